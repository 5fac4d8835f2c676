"""The integer binary64 <-> binary32 conversions (csrc/cvt.cuh) that the mixed V-cycle
applies to its FP64 input and FP32 result: on the host against the C++ conversions of
this machine (IEEE 754 round to nearest, ties to even), and on the GPU through the C ABI
(gf_round_to_f32, gf_widen_to_f64) against CUDA's own conversions, bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_conversions_match_ieee_on_the_host(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = tmp_path / "cvt_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", str(exe), os.path.join(HERE, "cvt", "cvt_check.cpp")],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout


def _edge_doubles():
    f32max = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    sub = 2.0 ** -149
    vals = [0.0, -0.0, 1.0, -1.0, f32max, np.nextafter(f32max, np.inf), f32max * (1 + 2.0 ** -24),
            f32max * (1 + 2.0 ** -25), 1e39, -1e39, np.inf, -np.inf, np.nan, tiny, np.nextafter(tiny, 0.0),
            sub, sub / 2, np.nextafter(sub / 2, 1.0), np.nextafter(sub / 2, 0.0), 3 * sub / 2, 5 * sub / 2,
            2.0 ** -160, 5e-324, -5e-324, 2.2250738585072014e-308, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24]
    return np.array(vals, dtype=np.float64)


@pytest.mark.gpu
def test_integer_conversions_match_cuda_bit_for_bit():
    torch = pytest.importorskip("torch")
    from paper_2607_26382_b300 import build
    build.build()
    import paper_2607_26382_b300 as gf

    g = torch.Generator(device="cuda").manual_seed(7)
    n = 1 << 22
    # random binary64 patterns (every exponent), patterns near the binary32 range with the
    # low 29 fraction bits at, just below and just above a tie, and the edges
    raw = torch.randint(-(2 ** 63), 2 ** 63 - 1, (n,), generator=g, device="cuda", dtype=torch.int64)
    near = raw[n // 2:].clone()
    expo = torch.randint(850, 1180, (near.numel(),), generator=g, device="cuda", dtype=torch.int64)
    near = (near & ~(0x7ff << 52)) | (expo << 52)
    low = torch.tensor([0x10000000, 0x0FFFFFFF, 0x10000001], device="cuda", dtype=torch.int64)
    pick = torch.randint(0, 4, (near.numel(),), generator=g, device="cuda")
    tie = (near & ~0x1FFFFFFF) | low[pick.clamp(max=2)]
    near = torch.where(pick < 3, tie, near)
    raw[n // 2:] = near
    x = torch.cat([raw.view(torch.float64), torch.as_tensor(_edge_doubles(), device="cuda")])
    got = gf.round_to_f32(x)
    ref = x.float()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(got), nan)
    assert torch.equal(got[~nan].view(torch.int32), ref[~nan].view(torch.int32))

    y = torch.randint(-(2 ** 31), 2 ** 31, (n,), generator=g, device="cuda", dtype=torch.int64).to(torch.int32)
    y[:4096] = torch.arange(1, 4097, device="cuda", dtype=torch.int32) * 97   # binary32 subnormals
    yf = torch.cat([y.view(torch.float32),
                    torch.tensor([0.0, -0.0, float("inf"), float("-inf"), float("nan")], device="cuda")])
    gotw = gf.widen_to_f64(yf)
    refw = yf.double()
    nanw = torch.isnan(refw)
    assert torch.equal(torch.isnan(gotw), nanw)
    assert torch.equal(gotw[~nanw].view(torch.int64), refw[~nanw].view(torch.int64))
    # n = 0 enqueues nothing
    assert gf.round_to_f32(x[:0]).numel() == 0
