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
// and beta = g_0 (.) scale.  The dense products run in the register-tiled GEMM
// below (FP32 for MALA_MIXED, FP64 for MALA_FP64_PLAIN, in the precision of the
// chain's tests); bias, activation, masks and the input scaling are the
// elementwise kernels below.
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

// ---- row GEMM: C[P][N] = X[P][K] op(W), op(W) = W^T (W [N][K]) or W (W [K][N]) ----
//
// A CTA of 256 threads (16 x 16) computes a BM x BN tile of C, each thread a
// contiguous TM x TN block (rows ty*TM.., columns tx*TN..), so a step of k
// reads its operands as 16-byte vectors from shared memory.  K advances in
// steps of BK through two shared-memory buffers: X as [BK][BM + pad] (the pad
// spreads the transposing stores over the banks and keeps rows 16-byte
// aligned), op(W) as [BK][BN]; the next step's tile is loaded into registers
// while the current one is multiplied.  Every output is one FMA chain over k in
// order, accumulated in T.
template <class T> struct GemmShape;
template <> struct GemmShape<float> { static constexpr int BM = 128, BN = 64, BK = 16, PAD = 4; };
template <> struct GemmShape<double> { static constexpr int BM = 64, BN = 64, BK = 16, PAD = 2; };

template <class T, bool TRANS>
__global__ void __launch_bounds__(256) k_gemm_rows(const T* __restrict__ X, const T* __restrict__ W, int64_t P, int N,
                                                   int K, T* __restrict__ Cm) {
    constexpr int BM = GemmShape<T>::BM, BN = GemmShape<T>::BN, BK = GemmShape<T>::BK, PAD = GemmShape<T>::PAD;
    constexpr int TM = BM / 16, TN = BN / 16;
    constexpr int VEC = 16 / sizeof(T);          // elements per 16-byte vector
    constexpr int XL = BM * BK / 256, WL = BN * BK / 256;  // tile elements a thread loads
    __shared__ __align__(16) T xs[2][BK][BM + PAD];
    __shared__ __align__(16) T ws[2][BK][BN];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    // the next K-tile travels global -> registers while the current one is multiplied
    T xr[XL], wr[WL];
    auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < XL; ++u) {  // X rows m0.., columns k0..k0+BK: consecutive threads along k
            const int idx = threadIdx.x + 256 * u;
            const int r = idx / BK, kk = idx - r * BK;
            const int64_t m = m0 + r;
            const int k = k0 + kk;
            xr[u] = (m < P && k < K) ? X[m * K + k] : T(0);
        }
#pragma unroll
        for (int u = 0; u < WL; ++u) {
            const int idx = threadIdx.x + 256 * u;
            int kk, c;
            if (TRANS) {  // W [N][K]: consecutive threads along k
                c = idx / BK;
                kk = idx - c * BK;
            } else {      // W [K][N]: consecutive threads along n
                kk = idx / BN;
                c = idx - kk * BN;
            }
            const int k = k0 + kk, n = n0 + c;
            wr[u] = (k < K && n < N) ? (TRANS ? W[(size_t)n * K + k] : W[(size_t)k * N + n]) : T(0);
        }
    };
    auto store = [&](int b) {
#pragma unroll
        for (int u = 0; u < XL; ++u) {
            const int idx = threadIdx.x + 256 * u;
            const int r = idx / BK, kk = idx - r * BK;
            xs[b][kk][r] = xr[u];
        }
#pragma unroll
        for (int u = 0; u < WL; ++u) {
            const int idx = threadIdx.x + 256 * u;
            int kk, c;
            if (TRANS) {
                c = idx / BK;
                kk = idx - c * BK;
            } else {
                kk = idx / BN;
                c = idx - kk * BN;
            }
            ws[b][kk][c] = wr[u];
        }
    };
    const int ntile = (K + BK - 1) / BK;
    load(0);
    store(0);
    __syncthreads();
    for (int t = 0; t < ntile; ++t) {
        const int b = t & 1;
        if (t + 1 < ntile) load((t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; i += VEC)
                *reinterpret_cast<uint4*>(&a[i]) = *reinterpret_cast<const uint4*>(&xs[b][kk][ty * TM + i]);
#pragma unroll
            for (int j = 0; j < TN; j += VEC)
                *reinterpret_cast<uint4*>(&bv[j]) = *reinterpret_cast<const uint4*>(&ws[b][kk][tx * TN + j]);
            if constexpr (sizeof(T) == 4) {
                // rows in pairs: one packed FP32x2 FMA per (row pair, column), each half the same
                // fused multiply-add as the scalar form (same bits), half the issue slots
#pragma unroll
                for (int i = 0; i < TM; i += 2)
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        const float2 r = __ffma2_rn(make_float2(a[i], a[i + 1]), make_float2(bv[j], bv[j]),
                                                    make_float2(acc[i][j], acc[i + 1][j]));
                        acc[i][j] = r.x;
                        acc[i + 1][j] = r.y;
                    }
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
            }
        }
        // the other buffer was last read before the previous barrier
        if (t + 1 < ntile) store(b ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t m = m0 + ty * TM + i;
        if (m >= P) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx * TN + j;
            if (n < N) Cm[m * N + n] = acc[i][j];
        }
    }
}

template <class T>
int gemm_rows(bool trans_w, int64_t P, int N, int K, const T* W, const T* X, T* Cm, cudaStream_t st) {
    constexpr int BM = GemmShape<T>::BM, BN = GemmShape<T>::BN;
    const int64_t gx = (P + BM - 1) / BM;
    if (gx > 0x7fffffff) return fail(MALA_ERR_UNSUPPORTED, "too many rows for the backward GEMM");
    const dim3 grid((unsigned)gx, (unsigned)((N + BN - 1) / BN));
    if (trans_w) k_gemm_rows<T, true><<<grid, 256, 0, st>>>(X, W, P, N, K, Cm);
    else k_gemm_rows<T, false><<<grid, 256, 0, st>>>(X, W, P, N, K, Cm);
    MALA_CUDA_TRY(cudaGetLastError());
    return MALA_OK;
}

template <class T>
int backward_impl(Ctx* c, const Model* m, const T* B, int64_t P, const double* v_dev, T* beta, cudaStream_t st) {
    const int nl = m->n_layers;
    const std::vector<int>& d = m->dims;
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
        MALA_PROF(c, "k_gemm_rows", st, MALA_TRY(gemm_rows<T>(true, P, d[l + 1], d[l], W[l], H[l], H[l + 1], st)));
        MALA_PROF(c, "k_bwd_elementwise", st,
                  (k_bias_act<T><<<ew_blocks(c, P * d[l + 1]), 256, 0, st>>>(H[l + 1], P, d[l + 1], bb[l], slope, 1)));
    }
    // dE/dH_{nl-1}: one vector u for a linear output layer, else per point in Gb[cur]
    bool vec = false;
    if (!m->activate_output) {
        k_vec_wt<T><<<(d[nl - 1] + 127) / 128, 128, 0, st>>>(m->Wd[nl - 1], v_dev, d[nl], d[nl - 1], u);
        vec = true;
    } else {
        MALA_PROF(c, "k_gemm_rows", st, MALA_TRY(gemm_rows<T>(true, P, d[nl], d[nl - 1], W[nl - 1], H[nl - 1], Zo, st)));
        MALA_PROF(c, "k_bwd_elementwise", st,
                  (k_bias_act<T><<<ew_blocks(c, P * d[nl]), 256, 0, st>>>(Zo, P, d[nl], bb[nl - 1], slope, 1)));
        k_cvt<T><<<ew_blocks(c, d[nl]), 256, 0, st>>>(v_dev, d[nl], u);
        MALA_PROF(c, "k_bwd_elementwise", st,
                  (k_mask<T><<<ew_blocks(c, P * d[nl]), 256, 0, st>>>(Zo, u, Zo, P, d[nl], slope)));
        MALA_PROF(c, "k_gemm_rows", st, MALA_TRY(gemm_rows<T>(false, P, d[nl - 1], d[nl], W[nl - 1], Zo, Gb[cur], st)));
    }
    for (int l = nl - 1; l >= 1; --l) {
        // delta = dE/dH_l (.) sigma'(z) (H_l = sigma(z) is layer l-1's output), then dE/dH_{l-1} = delta W_{l-1}
        MALA_PROF(c, "k_bwd_elementwise", st,
                  (k_mask<T><<<ew_blocks(c, P * d[l]), 256, 0, st>>>(Gb[cur], vec ? u : nullptr, H[l], P, d[l],
                                                                     slope)));
        vec = false;
        MALA_PROF(c, "k_gemm_rows", st,
                  MALA_TRY(gemm_rows<T>(false, P, d[l - 1], d[l], W[l - 1], Gb[cur], Gb[cur ^ 1], st)));
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



}  // namespace mala
