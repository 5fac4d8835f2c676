// Learned first-floor selector: MLP 6 -> 32 -> 32 -> 4 (tanh, softmax), FP32, with
// hand-written forward, backward and Adam kernels (included at the end of
// gf_lib.cu). Not in the paper: its counterpart there is the two-feature rule of
// Eq. (trigger). Inputs: [log10 r50, log10 r100, r100/r50, fraction of voxels at
// floor, mean rho_hat, std rho_hat]; output: index of the first ladder floor to
// try. The guard and the rest of the ladder stay the fallback.
//
// Parameters are one flat FP32 vector: W1 (32x6, [out][in]), b1, W2 (32x32), b2,
// W3 (4x32), b3 -- 1412 numbers. Training is deterministic: per-sample gradients
// are written out and summed over the minibatch in a fixed order.
#pragma once

namespace gf {

constexpr int MLP_IN = 6, MLP_H = 32, MLP_OUT = 4;
constexpr int MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_H * MLP_IN, MLP_W2 = MLP_B1 + MLP_H, MLP_B2 = MLP_W2 + MLP_H * MLP_H,
              MLP_W3 = MLP_B2 + MLP_H, MLP_B3 = MLP_W3 + MLP_OUT * MLP_H, MLP_P = MLP_B3 + MLP_OUT;

struct MLPNorm {
    float mu[MLP_IN];
    float inv_sd[MLP_IN];
};

__device__ __forceinline__ void mlp_forward_one(const float* __restrict__ th, const float* x, const MLPNorm& nm,
                                                float* z0, float* h1, float* h2, float* z3)
{
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) z0[i] = (x[i] - nm.mu[i]) * nm.inv_sd[i];
    for (int o = 0; o < MLP_H; ++o) {
        float s = th[MLP_B1 + o];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) s = fmaf(th[MLP_W1 + o * MLP_IN + i], z0[i], s);
        h1[o] = tanhf(s);
    }
    for (int o = 0; o < MLP_H; ++o) {
        float s = th[MLP_B2 + o];
        for (int i = 0; i < MLP_H; ++i) s = fmaf(th[MLP_W2 + o * MLP_H + i], h1[i], s);
        h2[o] = tanhf(s);
    }
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        float s = th[MLP_B3 + o];
        for (int i = 0; i < MLP_H; ++i) s = fmaf(th[MLP_W3 + o * MLP_H + i], h2[i], s);
        z3[o] = s;
    }
}

__global__ void __launch_bounds__(128)
mlp_forward_kernel(const float* __restrict__ theta, const float* __restrict__ X, int n, MLPNorm nm,
                   float* __restrict__ logits, int* __restrict__ cls)
{
    __shared__ float th[MLP_P];
    for (int p = threadIdx.x; p < MLP_P; p += blockDim.x) th[p] = theta[p];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float z0[MLP_IN], h1[MLP_H], h2[MLP_H], z3[MLP_OUT];
    mlp_forward_one(th, X + (long long)s * MLP_IN, nm, z0, h1, h2, z3);
    int best = 0;
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        if (logits) logits[(long long)s * MLP_OUT + o] = z3[o];
        if (z3[o] > z3[best]) best = o;
    }
    if (cls) cls[s] = best;
}

// Per-sample cross-entropy and its gradient (row s of gps, MLP_P floats), divided
// by the minibatch size nb so that the fixed-order sum is the mean gradient.
__global__ void __launch_bounds__(128)
mlp_grad_kernel(const float* __restrict__ theta, const float* __restrict__ X, const int* __restrict__ y,
                const int* __restrict__ idx, int nb, MLPNorm nm, float* __restrict__ gps, float* __restrict__ lps)
{
    __shared__ float th[MLP_P];
    for (int p = threadIdx.x; p < MLP_P; p += blockDim.x) th[p] = theta[p];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nb) return;
    const int r = idx ? idx[s] : s;
    float z0[MLP_IN], h1[MLP_H], h2[MLP_H], z3[MLP_OUT];
    mlp_forward_one(th, X + (long long)r * MLP_IN, nm, z0, h1, h2, z3);
    float mx = z3[0];
#pragma unroll
    for (int o = 1; o < MLP_OUT; ++o) mx = fmaxf(mx, z3[o]);
    float p[MLP_OUT], den = 0.f;
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        p[o] = expf(z3[o] - mx);
        den += p[o];
    }
    const int label = y[r];
    const float inv_nb = 1.0f / (float)nb;
    float d3[MLP_OUT];
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        p[o] /= den;
        d3[o] = (p[o] - (o == label ? 1.f : 0.f)) * inv_nb;
    }
    lps[s] = -logf(p[label]) * inv_nb;
    float* g = gps + (long long)s * MLP_P;
    float d2[MLP_H];
    for (int i = 0; i < MLP_H; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) acc = fmaf(d3[o], th[MLP_W3 + o * MLP_H + i], acc);
        d2[i] = acc * (1.f - h2[i] * h2[i]);
    }
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        for (int i = 0; i < MLP_H; ++i) g[MLP_W3 + o * MLP_H + i] = d3[o] * h2[i];
        g[MLP_B3 + o] = d3[o];
    }
    float d1[MLP_H];
    for (int i = 0; i < MLP_H; ++i) {
        float acc = 0.f;
        for (int o = 0; o < MLP_H; ++o) acc = fmaf(d2[o], th[MLP_W2 + o * MLP_H + i], acc);
        d1[i] = acc * (1.f - h1[i] * h1[i]);
    }
    for (int o = 0; o < MLP_H; ++o) {
        for (int i = 0; i < MLP_H; ++i) g[MLP_W2 + o * MLP_H + i] = d2[o] * h1[i];
        g[MLP_B2 + o] = d2[o];
    }
    for (int o = 0; o < MLP_H; ++o) {
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) g[MLP_W1 + o * MLP_IN + i] = d1[o] * z0[i];
        g[MLP_B1 + o] = d1[o];
    }
}

// grad[p] = sum_s gps[s][p] in sample order; loss likewise (thread MLP_P).
__global__ void mlp_reduce_kernel(const float* __restrict__ gps, const float* __restrict__ lps, int nb,
                                  float* __restrict__ grad, float* __restrict__ loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < MLP_P) {
        float s = 0.f;
        for (int q = 0; q < nb; ++q) s += gps[(long long)q * MLP_P + p];
        grad[p] = s;
    } else if (p == MLP_P) {
        float s = 0.f;
        for (int q = 0; q < nb; ++q) s += lps[q];
        *loss = s;
    }
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_P) return;
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp;
    const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    theta[p] -= lr * (mp / bc1) / (sqrtf(vp / bc2) + eps);
}

}  // namespace gf

struct gf_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    float *gps = nullptr, *lps = nullptr;
    int cap = 0;
    int* idx = nullptr;
    int idx_cap = 0;
    float* feat = nullptr;    // inference scratch (up to 4096 rows)
    int* cls = nullptr;
    float* logits = nullptr;
    long long t = 0;
    gf::MLPNorm norm{};
};

namespace {

int mlp_ensure(gf_mlp* M, int nb)
{
    if (nb <= M->cap) return GF_OK;
    cudaFree(M->gps);
    cudaFree(M->lps);
    M->gps = M->lps = nullptr;
    M->cap = 0;
    CK(cudaMalloc(&M->gps, sizeof(float) * (size_t)nb * gf::MLP_P));
    CK(cudaMalloc(&M->lps, sizeof(float) * (size_t)nb));
    M->cap = nb;
    return GF_OK;
}

// Host features (double) -> class per row, on the GPU.
int mlp_predict_host(gf_mlp* M, const double* feat, int n, int* cls)
{
    if (n > 4096) return set_err(GF_ERR_ARG, "at most 4096 rows per prediction");
    std::vector<float> f((size_t)n * gf::MLP_IN);
    for (size_t i = 0; i < f.size(); ++i) f[i] = (float)feat[i];
    CK(cudaMemcpyAsync(M->feat, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice, M->stream));
    gf::mlp_forward_kernel<<<(n + 127) / 128, 128, 0, M->stream>>>(M->theta, M->feat, n, M->norm, nullptr, M->cls);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(cls, M->cls, sizeof(int) * n, cudaMemcpyDeviceToHost, M->stream));
    CK(cudaStreamSynchronize(M->stream));
    return GF_OK;
}

// Softmax probabilities for host feature rows (n <= 4096).
int mlp_probs_host(gf_mlp* M, const double* feat, int n, double* probs)
{
    if (n > 4096) return set_err(GF_ERR_ARG, "at most 4096 rows per prediction");
    std::vector<float> f((size_t)n * gf::MLP_IN), lg((size_t)n * gf::MLP_OUT);
    for (size_t i = 0; i < f.size(); ++i) f[i] = (float)feat[i];
    CK(cudaMemcpyAsync(M->feat, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice, M->stream));
    gf::mlp_forward_kernel<<<(n + 127) / 128, 128, 0, M->stream>>>(M->theta, M->feat, n, M->norm, M->logits,
                                                                   nullptr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(lg.data(), M->logits, sizeof(float) * lg.size(), cudaMemcpyDeviceToHost, M->stream));
    CK(cudaStreamSynchronize(M->stream));
    for (int r = 0; r < n; ++r) {
        double mx = lg[r * gf::MLP_OUT];
        for (int o = 1; o < gf::MLP_OUT; ++o) mx = std::max(mx, (double)lg[r * gf::MLP_OUT + o]);
        double den = 0.0;
        for (int o = 0; o < gf::MLP_OUT; ++o) den += std::exp((double)lg[r * gf::MLP_OUT + o] - mx);
        for (int o = 0; o < gf::MLP_OUT; ++o) probs[r * gf::MLP_OUT + o] = std::exp((double)lg[r * gf::MLP_OUT + o] - mx) / den;
    }
    return GF_OK;
}

// First floor from the selector: argmax (c == 0) or the highest k with
// P(first admissible floor >= k) >= c.
int mlp_first_floors(gf_mlp* M, const double* feat, int n, double c, int nf, int* first)
{
    if (c <= 0.0) {
        RET(mlp_predict_host(M, feat, n, first));
    } else {
        std::vector<double> p((size_t)n * gf::MLP_OUT);
        RET(mlp_probs_host(M, feat, n, p.data()));
        for (int r = 0; r < n; ++r) {
            int k = 0;
            double tail = 0.0;
            for (int q = gf::MLP_OUT - 1; q >= 1; --q) {
                tail += p[r * gf::MLP_OUT + q];
                if (tail >= c) {
                    k = q;
                    break;
                }
            }
            first[r] = k;
        }
    }
    for (int r = 0; r < n; ++r) first[r] = std::min(std::max(first[r], 0), nf - 1);
    return GF_OK;
}

}  // namespace

extern "C" {

int gf_mlp_probs(gf_mlp* M, const double* feat, int n, double* probs)
{
    if (!M || !feat || !probs || n < 1) return set_err(GF_ERR_ARG, "bad argument");
    return mlp_probs_host(M, feat, n, probs);
}

int gf_mlp_create(const float* theta0, void* stream, gf_mlp** out)
{
    if (!out || !theta0) return set_err(GF_ERR_ARG, "null pointer");
    gf_mlp* M = new gf_mlp();
    M->stream = (cudaStream_t)stream;
    auto fail = [&](int code) { gf_mlp_destroy(M); return code; };
    if (cudaGetDevice(&M->device) != cudaSuccess) return fail(set_err(GF_ERR_CUDA, "cudaGetDevice"));
    const size_t P = sizeof(float) * gf::MLP_P;
    if (cudaMalloc(&M->theta, P) != cudaSuccess || cudaMalloc(&M->m, P) != cudaSuccess ||
        cudaMalloc(&M->v, P) != cudaSuccess || cudaMalloc(&M->grad, P) != cudaSuccess ||
        cudaMalloc(&M->loss, sizeof(float)) != cudaSuccess ||
        cudaMalloc(&M->feat, sizeof(float) * 4096 * gf::MLP_IN) != cudaSuccess ||
        cudaMalloc(&M->cls, sizeof(int) * 4096) != cudaSuccess ||
        cudaMalloc(&M->logits, sizeof(float) * 4096 * gf::MLP_OUT) != cudaSuccess)
        return fail(set_err(GF_ERR_OOM, "mlp buffers"));
    if (cudaMemcpy(M->theta, theta0, P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(M->m, 0, P) != cudaSuccess || cudaMemset(M->v, 0, P) != cudaSuccess)
        return fail(set_err(GF_ERR_CUDA, "mlp init"));
    for (int i = 0; i < gf::MLP_IN; ++i) {
        M->norm.mu[i] = 0.f;
        M->norm.inv_sd[i] = 1.f;
    }
    *out = M;
    return GF_OK;
}

int gf_mlp_destroy(gf_mlp* M)
{
    if (!M) return GF_OK;
    cudaFree(M->theta); cudaFree(M->m); cudaFree(M->v); cudaFree(M->grad); cudaFree(M->loss);
    cudaFree(M->gps); cudaFree(M->lps); cudaFree(M->idx); cudaFree(M->feat); cudaFree(M->cls);
    cudaFree(M->logits);
    delete M;
    return GF_OK;
}

int gf_mlp_set_norm(gf_mlp* M, const float* mu, const float* sd)
{
    if (!M || !mu || !sd) return set_err(GF_ERR_ARG, "null pointer");
    for (int i = 0; i < gf::MLP_IN; ++i) {
        if (!(sd[i] > 0.f)) return set_err(GF_ERR_ARG, "sd must be > 0");
        M->norm.mu[i] = mu[i];
        M->norm.inv_sd[i] = 1.f / sd[i];
    }
    return GF_OK;
}

int gf_mlp_get_params(gf_mlp* M, float* theta)
{
    if (!M || !theta) return set_err(GF_ERR_ARG, "null pointer");
    CK(cudaStreamSynchronize(M->stream));
    CK(cudaMemcpy(theta, M->theta, sizeof(float) * gf::MLP_P, cudaMemcpyDeviceToHost));
    return GF_OK;
}

int gf_mlp_forward(gf_mlp* M, const float* X, int n, float* logits)
{
    if (!M || !X || !logits || n < 0) return set_err(GF_ERR_ARG, "bad argument");
    if (n == 0) return GF_OK;
    gf::mlp_forward_kernel<<<(n + 127) / 128, 128, 0, M->stream>>>(M->theta, X, n, M->norm, logits, nullptr);
    CK(cudaGetLastError());
    return GF_OK;
}

int gf_mlp_loss_grad(gf_mlp* M, const float* X, const int* y, int n, float* loss, float* grad)
{
    if (!M || !X || !y || !loss || !grad || n < 1) return set_err(GF_ERR_ARG, "bad argument");
    RET(mlp_ensure(M, n));
    gf::mlp_grad_kernel<<<(n + 127) / 128, 128, 0, M->stream>>>(M->theta, X, y, nullptr, n, M->norm, M->gps, M->lps);
    CK(cudaGetLastError());
    gf::mlp_reduce_kernel<<<(gf::MLP_P + 1 + 255) / 256, 256, 0, M->stream>>>(M->gps, M->lps, n, M->grad, M->loss);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, M->stream));
    CK(cudaMemcpyAsync(grad, M->grad, sizeof(float) * gf::MLP_P, cudaMemcpyDeviceToHost, M->stream));
    CK(cudaStreamSynchronize(M->stream));
    return GF_OK;
}

int gf_mlp_train(gf_mlp* M, const float* X, const int* y, int n, const int* perm, int epochs, int batch,
                 float lr, float* final_loss)
{
    if (!M || !X || !y || n < 1 || epochs < 0 || batch < 1) return set_err(GF_ERR_ARG, "bad argument");
    const int nb = std::min(batch, n);
    RET(mlp_ensure(M, nb));
    const long long total = (long long)epochs * n;
    if (perm && total > M->idx_cap) {
        cudaFree(M->idx);
        M->idx = nullptr;
        M->idx_cap = 0;
        CK(cudaMalloc(&M->idx, sizeof(int) * total));
        M->idx_cap = (int)total;
    }
    if (perm) CK(cudaMemcpyAsync(M->idx, perm, sizeof(int) * total, cudaMemcpyHostToDevice, M->stream));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < epochs; ++e) {
        for (int s0 = 0; s0 + nb <= n; s0 += nb) {   // full minibatches only
            const int* idx = perm ? M->idx + (long long)e * n + s0 : nullptr;
            const float* Xs = perm ? X : X + (long long)s0 * gf::MLP_IN;
            const int* ys = perm ? y : y + s0;
            gf::mlp_grad_kernel<<<(nb + 127) / 128, 128, 0, M->stream>>>(M->theta, Xs, ys, idx, nb, M->norm, M->gps,
                                                                         M->lps);
            gf::mlp_reduce_kernel<<<(gf::MLP_P + 1 + 255) / 256, 256, 0, M->stream>>>(M->gps, M->lps, nb, M->grad,
                                                                                     M->loss);
            M->t += 1;
            const float bc1 = 1.f - powf(b1, (float)M->t), bc2 = 1.f - powf(b2, (float)M->t);
            gf::adam_kernel<<<(gf::MLP_P + 255) / 256, 256, 0, M->stream>>>(M->theta, M->m, M->v, M->grad, lr, b1, b2,
                                                                            eps, bc1, bc2);
            CK(cudaGetLastError());
        }
    }
    if (final_loss) {
        CK(cudaMemcpyAsync(final_loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, M->stream));
    }
    CK(cudaStreamSynchronize(M->stream));
    return GF_OK;
}

int gf_mlp_predict(gf_mlp* M, const double* feat, int n, int* cls)
{
    if (!M || !feat || !cls || n < 1) return set_err(GF_ERR_ARG, "bad argument");
    return mlp_predict_host(M, feat, n, cls);
}

}  // extern "C"
