// mlp_bwd.cu -- the network's vector-Jacobian product, the second factor of
// Eq. forcesmala applied to the vector v = dE/d LDOS(r, .):
//     beta(r, :) = sum_e v_e d LDOS(r, e) / d B(r, :)
// for the feed-forward network of Eq. ffnn (LeakyReLU hidden layers, optional
// input standardisation h_0 = (B - shift) * scale).
//
// The upstream vector is the same at every grid point (dE_b/dLDOS(r, e) =
// dV dE_b/dD_e), so for a linear output layer the first backward step is one
// vector u = W_L^T v shared by all points.  The hidden pre-activations are
// recomputed (the forward pass of the LDOS keeps none), then
//     delta_l = g_l (.) sigma'(z_l),  g_{l-1} = delta_l W_l,
// with sigma'(z) read from the sign of h = sigma(z) (LeakyReLU keeps the sign),
// and beta = g_0 (.) scale.  The dense products run as cuBLAS GEMMs (FP32 for
// MALA_MIXED, FP64 for MALA_FP64_PLAIN); bias, activation, masks and the input
// scaling are the elementwise kernels below.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "mala_internal.h"

namespace mala {

namespace {

template <class T>
__global__ void k_in_std(const T* __restrict__ B, int64_t P, int K, const T* __restrict__ shift,
                         const T* __restrict__ scale, T* __restrict__ H) {
    const int64_t n = P * K;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        H[i] = (B[i] - shift[k]) * scale[k];
    }
}

template <class T>
__global__ void k_bias_act(T* __restrict__ Z, int64_t P, int N, const T* __restrict__ b, T slope, int act) {
    const int64_t n = P * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T z = Z[i] + b[i % N];
        if (act) z = z > T(0) ? z : slope * z;
        Z[i] = z;
    }
}

// G[p][k] = (vec ? u[k] : G[p][k]) * (H[p][k] > 0 ? 1 : slope)
template <class T>
__global__ void k_mask(T* __restrict__ G, const T* __restrict__ u, const T* __restrict__ H, int64_t P, int N, T slope) {
    const int64_t n = P * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T g = u ? u[i % N] : G[i];
        G[i] = H[i] > T(0) ? g : slope * g;
    }
}

// beta[p][k] = (vec ? u[k] : G[p][k]) * scale[k]
template <class T>
__global__ void k_out_scale(const T* __restrict__ G, const T* __restrict__ u, const T* __restrict__ scale, int64_t P,
                            int K, T* __restrict__ beta) {
    const int64_t n = P * K;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        beta[i] = (u ? u[k] : G[i]) * scale[k];
    }
}

// u[k] = sum_n W[n][k] v[n] (W [N][K] row-major), FP64 accumulation
template <class T>
__global__ void k_vec_wt(const double* __restrict__ W, const double* __restrict__ v, int N, int K, T* __restrict__ u) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double s = 0.0;
    for (int n = 0; n < N; ++n) s += W[(size_t)n * K + k] * v[n];
    u[k] = (T)s;
}

template <class T>
__global__ void k_cvt(const double* __restrict__ x, int64_t n, T* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (T)x[i];
}

unsigned ew_blocks(Ctx* c, int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 32));
}

// C[P][N] (row-major) = X[P][K] W^T (W [N][K] row-major), or with trans_w = false C[P][N] = X[P][K] W (W [K][N])
cublasStatus_t gemm_rows(cublasHandle_t h, bool trans_w, int64_t P, int N, int K, const float* W, const float* X,
                         float* Cm) {
    const float one = 1.f, zero = 0.f;
    return cublasSgemm(h, trans_w ? CUBLAS_OP_T : CUBLAS_OP_N, CUBLAS_OP_N, N, (int)P, K, &one, W, trans_w ? K : N, X,
                       K, &zero, Cm, N);
}
cublasStatus_t gemm_rows(cublasHandle_t h, bool trans_w, int64_t P, int N, int K, const double* W, const double* X,
                         double* Cm) {
    const double one = 1.0, zero = 0.0;
    return cublasDgemm(h, trans_w ? CUBLAS_OP_T : CUBLAS_OP_N, CUBLAS_OP_N, N, (int)P, K, &one, W, trans_w ? K : N, X,
                       K, &zero, Cm, N);
}

template <class T>
int backward_impl(Ctx* c, const Model* m, const T* B, int64_t P, const double* v_dev, T* beta, cudaStream_t st) {
    const int nl = m->n_layers;
    const std::vector<int>& d = m->dims;
    if (!c->cublas) {
        cublasHandle_t h = nullptr;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return fail(MALA_ERR_CUDA, "cublasCreate failed");
        c->cublas = h;
    }
    cublasHandle_t h = static_cast<cublasHandle_t>(c->cublas);
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return fail(MALA_ERR_CUDA, "cublasSetStream failed");
    // parameters in T: W_l [d_{l+1}][d_l], b_l, shift, scale; then the vector u
    size_t npar = 2 * (size_t)d[0];
    for (int l = 0; l < nl; ++l) npar += (size_t)d[l] * d[l + 1] + d[l + 1];
    int wmax = 1;
    for (int l = 0; l <= nl; ++l) wmax = std::max(wmax, d[l]);
    MALA_TRY(c->ws_force_mlp.reserve(c, sizeof(T) * (npar + wmax + 64 * (size_t)(nl + 3))));
    T* par = c->ws_force_mlp.as<T>();
    std::vector<T*> W(nl), bb(nl);
    size_t o = 0;
    auto take = [&](size_t n) {
        T* p = par + o;
        o += (n + 63) & ~size_t(63);
        return p;
    };
    T* shift = take(d[0]);
    T* scale = take(d[0]);
    for (int l = 0; l < nl; ++l) {
        W[l] = take((size_t)d[l] * d[l + 1]);
        bb[l] = take(d[l + 1]);
    }
    T* u = take(wmax);
    if constexpr (sizeof(T) == 8) {
        MALA_CUDA_TRY(cudaMemcpyAsync(shift, m->in_shift_d, sizeof(double) * d[0], cudaMemcpyDeviceToDevice, st));
        MALA_CUDA_TRY(cudaMemcpyAsync(scale, m->in_scale_d, sizeof(double) * d[0], cudaMemcpyDeviceToDevice, st));
        for (int l = 0; l < nl; ++l) {
            MALA_CUDA_TRY(cudaMemcpyAsync(W[l], m->Wd[l], sizeof(double) * d[l] * d[l + 1], cudaMemcpyDeviceToDevice, st));
            MALA_CUDA_TRY(cudaMemcpyAsync(bb[l], m->bd[l], sizeof(double) * d[l + 1], cudaMemcpyDeviceToDevice, st));
        }
    } else {
        k_cvt<T><<<ew_blocks(c, d[0]), 256, 0, st>>>(m->in_shift_d, d[0], shift);
        k_cvt<T><<<ew_blocks(c, d[0]), 256, 0, st>>>(m->in_scale_d, d[0], scale);
        for (int l = 0; l < nl; ++l) {
            k_cvt<T><<<ew_blocks(c, (int64_t)d[l] * d[l + 1]), 256, 0, st>>>(m->Wd[l], (int64_t)d[l] * d[l + 1], W[l]);
            k_cvt<T><<<ew_blocks(c, d[l + 1]), 256, 0, st>>>(m->bd[l], d[l + 1], bb[l]);
        }
    }
    MALA_CUDA_TRY(cudaGetLastError());
    if (P <= 0) return MALA_OK;
    // activations H_0 .. H_{nl-1} (kept: their signs are the masks), two gradient
    // buffers [P][wmax] (a GEMM cannot write over its input) and, with an activated
    // output layer, its outputs
    size_t acts = 0;
    for (int l = 0; l < nl; ++l) acts += (size_t)d[l];
    const size_t per_row = acts + 2 * (size_t)wmax + (m->activate_output ? (size_t)d[nl] : 0);
    MALA_TRY(c->ws_force_beta.reserve(c, sizeof(T) * (size_t)P * per_row + 256));
    std::vector<T*> H(nl);
    T* base = c->ws_force_beta.as<T>();
    for (int l = 0; l < nl; ++l) {
        H[l] = base;
        base += (size_t)P * d[l];
    }
    T* Gb[2] = {base, base + (size_t)P * wmax};
    T* Zo = base + 2 * (size_t)P * wmax;
    int cur = 0;
    const T slope = (T)m->slope_d;
    MALA_PROF(c, "k_bwd_elementwise", st,
              (k_in_std<T><<<ew_blocks(c, P * d[0]), 256, 0, st>>>(B, P, d[0], shift, scale, H[0])));
    for (int l = 0; l + 1 < nl; ++l) {
        if (gemm_rows(h, true, P, d[l + 1], d[l], W[l], H[l], H[l + 1]) != CUBLAS_STATUS_SUCCESS)
            return fail(MALA_ERR_CUDA, "cuBLAS GEMM (layer %d forward) failed", l);
        MALA_PROF(c, "k_bwd_elementwise", st,
                  (k_bias_act<T><<<ew_blocks(c, P * d[l + 1]), 256, 0, st>>>(H[l + 1], P, d[l + 1], bb[l], slope, 1)));
    }
    // dE/dH_{nl-1}: one vector u for a linear output layer, else per point in Gb[cur]
    bool vec = false;
    if (!m->activate_output) {
        k_vec_wt<T><<<(d[nl - 1] + 127) / 128, 128, 0, st>>>(m->Wd[nl - 1], v_dev, d[nl], d[nl - 1], u);
        vec = true;
    } else {
        if (gemm_rows(h, true, P, d[nl], d[nl - 1], W[nl - 1], H[nl - 1], Zo) != CUBLAS_STATUS_SUCCESS)
            return fail(MALA_ERR_CUDA, "cuBLAS GEMM (output layer) failed");
        MALA_PROF(c, "k_bwd_elementwise", st,
                  (k_bias_act<T><<<ew_blocks(c, P * d[nl]), 256, 0, st>>>(Zo, P, d[nl], bb[nl - 1], slope, 1)));
        k_cvt<T><<<ew_blocks(c, d[nl]), 256, 0, st>>>(v_dev, d[nl], u);
        MALA_PROF(c, "k_bwd_elementwise", st,
                  (k_mask<T><<<ew_blocks(c, P * d[nl]), 256, 0, st>>>(Zo, u, Zo, P, d[nl], slope)));
        if (gemm_rows(h, false, P, d[nl - 1], d[nl], W[nl - 1], Zo, Gb[cur]) != CUBLAS_STATUS_SUCCESS)
            return fail(MALA_ERR_CUDA, "cuBLAS GEMM (output layer backward) failed");
    }
    for (int l = nl - 1; l >= 1; --l) {
        // delta = dE/dH_l (.) sigma'(z) (H_l = sigma(z) is layer l-1's output), then dE/dH_{l-1} = delta W_{l-1}
        MALA_PROF(c, "k_bwd_elementwise", st,
                  (k_mask<T><<<ew_blocks(c, P * d[l]), 256, 0, st>>>(Gb[cur], vec ? u : nullptr, H[l], P, d[l],
                                                                     slope)));
        vec = false;
        if (gemm_rows(h, false, P, d[l - 1], d[l], W[l - 1], Gb[cur], Gb[cur ^ 1]) != CUBLAS_STATUS_SUCCESS)
            return fail(MALA_ERR_CUDA, "cuBLAS GEMM (layer %d backward) failed", l - 1);
        cur ^= 1;
    }
    T* G = Gb[cur];
    MALA_PROF(c, "k_bwd_elementwise", st,
              (k_out_scale<T><<<ew_blocks(c, P * d[0]), 256, 0, st>>>(G, vec ? u : nullptr, scale, P, d[0], beta)));
    MALA_CUDA_TRY(cudaGetLastError());
    return MALA_OK;
}

}  // namespace

int mlp_backward(Ctx* c, const Model* m, const void* B, int64_t P, const double* v_dev, void* beta,
                 mala_precision prec, cudaStream_t st) {
    if (prec == MALA_MIXED)
        return backward_impl<float>(c, m, static_cast<const float*>(B), P, v_dev, static_cast<float*>(beta), st);
    return backward_impl<double>(c, m, static_cast<const double*>(B), P, v_dev, static_cast<double*>(beta), st);
}

void cublas_release(Ctx* c) {
    if (c->cublas) cublasDestroy(static_cast<cublasHandle_t>(c->cublas));
    c->cublas = nullptr;
}

}  // namespace mala
