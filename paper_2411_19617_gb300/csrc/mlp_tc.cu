// mlp_tc.cu -- the per-point feed-forward network (paper Eq. ffnn,
// x_{l+1} = act(W_l x_l + b_l)) on the 5th-generation tensor cores, plus the
// FP64 path.
//
// MIXED path: a persistent kernel, one CTA of 8 warps per SM, walking tiles of
// 128 grid points (M = 128):
//   * the descriptors B[P][n_B] (FP32) of a tile are read row by row
//     (coalesced), standardised ((B - shift) * scale), rounded to BF16 and
//     written to shared memory in the UMMA K-major layout with the 128-byte
//     swizzle (the layout TMA produces with SWIZZLE_128B);
//   * every layer is a chain of tcgen05.mma (kind::f16, BF16 x BF16 -> FP32)
//     issued by one thread into a tensor-memory accumulator D[128][N] (one TMEM
//     lane per point); the layer's weights W_l[N][K] stream through two
//     shared-memory stages in K-blocks of 64 by TMA: block kb+1 is fetched
//     while the MMAs of block kb run, and the first two blocks of the next
//     layer (or of the next tile's first layer) are fetched while the
//     epilogue runs;
//   * the epilogue reads D with tcgen05.ld (thread = point, the two warps that
//     share a TMEM lane quarter take alternate 32-column chunks), adds the
//     bias, applies LeakyReLU on hidden layers and writes the BF16 activations
//     back to shared memory as the next layer's A operand;
//   * the last epilogue writes the LDOS in BF16 and, from the same rounded
//     values, adds the tile's column sums sum_r LDOS(r, xi) to the CTA's FP64
//     DOS partial; the partials of all CTAs are summed in CTA order afterwards,
//     so the DOS does not depend on timing.
// Every wait on an mbarrier is bounded (about one second of clock cycles); on
// expiry the kernel records an error code, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "mala_internal.h"

namespace mala {

namespace {

constexpr int kMlpThreads = 256;
constexpr int kMaxLayers = 4;
constexpr int kKBlk = 64;             // K elements per swizzle block (128 bytes of BF16)
constexpr int kMaxHiddenPad = 448;    // widest K of a hidden activation (7 blocks)
constexpr int kMaxNPad = 400;         // widest layer output held in one W stage
constexpr int kHBytes = 128 * kMaxHiddenPad * 2;  // 114688
constexpr int kStageBytes = kMaxNPad * 128;        // 51200: [N rows][64 K] BF16
constexpr int kMaxNE = 256;                        // widest output layer
constexpr int kSmemBytes = kHBytes + 2 * kStageBytes + 1024 /* barriers, tmem slot */ + kMaxNE * 8 /* DOS partial */ +
                           1024 /* alignment */;
constexpr long long kWaitCycles = 2000000000LL;

struct LayerDev {
    int K, Kpad, N, Npad, nkb;  // nkb = Kpad / 64
    int boxN;                   // TMA box rows (Npad split in <= 256-row boxes)
    int act;                    // apply LeakyReLU
    const float* bias;          // [Npad]
};

struct MlpParams {
    int n_layers;
    LayerDev L[kMaxLayers];
    float slope;
    int nB;                 // descriptor count (K of layer 0)
    const float* B;         // [P][nB]
    const float* shift;     // [nB]
    const float* scale;     // [nB]
    __nv_bfloat16* ldos;    // [P][N_E]
    double* cta_dos;        // [gridDim.x][N_E] or nullptr
    int64_t P;
    int* err;
};

struct TMaps {
    CUtensorMap m[kMaxLayers];
};

// ---- PTX wrappers ---------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait; false (and *err set) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, int* err, int code) {
    const long long t0 = clock64();
    while (!mbar_try(bar, phase)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                   // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // SBO
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// byte offset of element (row r, k) in a [128][64] BF16 K-block with the
// 128-byte swizzle (16-byte chunk index XOR row % 8)
__device__ __forceinline__ uint32_t swz(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// tcgen05.ld of 32 consecutive columns of the warp's TMEM lane quarter.  The
// registers are valid only after tmem_wait(), which names them as operands so
// that no use can be scheduled ahead of the wait.
__device__ __forceinline__ void tmem_issue32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr + 16u));
}

__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                   "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]),
                   "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// bias + activation of 32 accumulator columns c0.. (zero beyond the layer's N)
__device__ __forceinline__ void bias_act32(const uint32_t (&r)[32], float (&x)[32], int c0, const LayerDev& L,
                                           float slope) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c0 + 4 * q < L.Npad) b = __ldg(reinterpret_cast<const float4*>(L.bias) + (c0 / 4 + q));
        const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = c0 + 4 * q + i;
            float t = (c < L.N) ? __uint_as_float(r[4 * q + i]) + bb[i] : 0.f;
            if (L.act) t = t > 0.f ? t : slope * t;
            x[4 * q + i] = t;
        }
    }
}

// Weight pipeline state of the issuing thread.  Stage s holds K-block kb with
// kb % 2 == s.  full[s] completes when a stage's TMA bytes have landed,
// free[s] when the MMAs that read it have finished; every completion of either
// is waited exactly once, in order, before the barrier can complete again.
struct WPipe {
    uint32_t full[2], free_[2];
    uint32_t ph_full[2] = {0, 0}, ph_free[2] = {0, 0};
    bool pend[2] = {false, false};      // a free[s] completion not yet waited for
    bool inflight[2] = {false, false};  // a full[s] completion not yet waited for
};

__device__ __forceinline__ bool wait_full(WPipe& wp, int s, int* err) {
    const bool ok = mbar_wait(wp.full[s], wp.ph_full[s], err, 2);
    wp.ph_full[s] ^= 1;
    wp.inflight[s] = false;
    return ok;
}

__device__ __forceinline__ bool load_stage(WPipe& wp, const CUtensorMap* map, const LayerDev& L, int kb,
                                           unsigned char* sW, int* err) {
    const int s = kb & 1;
    if (wp.pend[s]) {
        if (!mbar_wait(wp.free_[s], wp.ph_free[s], err, 3)) return false;
        wp.ph_free[s] ^= 1;
        wp.pend[s] = false;
    }
    mbar_expect_tx(wp.full[s], (uint32_t)L.Npad * 128u);
    wp.inflight[s] = true;
    for (int n0 = 0; n0 < L.Npad; n0 += L.boxN)
        tma_load_2d(smem_u32(sW + s * kStageBytes + n0 * 128), map, kb * kKBlk, n0, wp.full[s]);
    return true;
}

__global__ void __launch_bounds__(kMlpThreads, 1) k_mlp_tc(const __grid_constant__ TMaps maps, MlpParams prm) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sH = sm;                          // activations, K-blocks of [128][64] BF16
    unsigned char* sW = sm + kHBytes;                // two weight stages
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kHBytes + 2 * kStageBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 8);
    double* sDos = reinterpret_cast<double*>(sm + kHBytes + 2 * kStageBytes + 1024);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;  // TMEM lane quarter, column-chunk parity
    const int64_t ntiles = (prm.P + 127) / 128;
    const int NE = prm.L[prm.n_layers - 1].N;
    WPipe wp;
    wp.full[0] = smem_u32(&bars[0]);
    wp.full[1] = smem_u32(&bars[1]);
    wp.free_[0] = smem_u32(&bars[2]);
    wp.free_[1] = smem_u32(&bars[3]);
    const uint32_t bar_done = smem_u32(&bars[4]);

    if (tid == 0) {
        for (int i = 0; i < 5; ++i) mbar_init(smem_u32(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int l = 0; l < prm.n_layers; ++l)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.m[l])) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int c = tid; c < NE; c += kMlpThreads) sDos[c] = 0.0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t ph_done = 0;
    bool ok = true;
    if (tid == 0 && (int64_t)blockIdx.x < ntiles) {
        for (int kb = 0; kb < min(2, prm.L[0].nkb) && ok; ++kb) ok = load_stage(wp, &maps.m[0], prm.L[0], kb, sW, prm.err);
    }

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * 128;
        const int nrows = (int)min((int64_t)128, prm.P - row0);
        // ---- input tile: (B - shift) * scale -> BF16, swizzled, zero-padded ----
        // warp w takes rows 4w..4w+3 (+32 per pass), lane k = lane + 32 j;
        // up to 16 loads per thread are in flight before the first store
        {
            const int K0pad = prm.L[0].Kpad;
            const int nch = K0pad / 32;
            const float* __restrict__ src = prm.B + row0 * prm.nB;
            for (int rb = warp * 4; rb < 128; rb += 4 * (kMlpThreads / 32)) {
                for (int j0 = 0; j0 < nch; j0 += 4) {
                    float v[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int k = lane + 32 * (j0 + j);
                            v[i][j] = (k < prm.nB && rb + i < nrows) ? __ldg(src + (int64_t)(rb + i) * prm.nB + k) : 0.f;
                        }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (j0 + j >= nch) break;
                        const int k = lane + 32 * (j0 + j);
                        const bool in = k < prm.nB;
                        const float sh = in ? __ldg(prm.shift + k) : 0.f;
                        const float sc = in ? __ldg(prm.scale + k) : 0.f;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            *reinterpret_cast<__nv_bfloat16*>(sH + (k / kKBlk) * (128 * 128) + swz(rb + i, k % kKBlk)) =
                                __float2bfloat16_rn((v[i][j] - sh) * sc);
                    }
                }
            }
            // warm L2 with the next tile's descriptors (a hint; skipped when unaligned)
            if (tid == 32) {
                const int64_t nt = tile + gridDim.x;
                if (nt < ntiles) {
                    const int64_t nr = min((int64_t)128, prm.P - nt * 128);
                    const float* nsrc = prm.B + nt * 128 * prm.nB;
                    const uint32_t bytes = (uint32_t)(nr * prm.nB * 4) & ~15u;
                    if ((reinterpret_cast<uintptr_t>(nsrc) & 15) == 0 && bytes > 0)
                        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(nsrc), "r"(bytes) : "memory");
                }
            }
        }
        fence_proxy_async();
        tc_fence_before();
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        tc_fence_after();

        for (int l = 0; l < prm.n_layers; ++l) {
            const LayerDev& L = prm.L[l];
            // ---- MMA chain of layer l (one thread issues, the rest wait) ----
            if (tid == 0) {
                for (int kb = 0; kb < L.nkb && ok; ++kb) {
                    const int s = kb & 1;
                    ok = wait_full(wp, s, prm.err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(sH + kb * (128 * 128));
                    const uint32_t b_base = smem_u32(sW + s * kStageBytes);
#pragma unroll
                    for (int k = 0; k < kKBlk / 16; ++k) {
                        for (int n0 = 0; n0 < L.Npad; n0 += 256) {
                            const int nn = min(256, L.Npad - n0);
                            mma_bf16(tmem + (uint32_t)n0, sdesc(a_base + k * 32), sdesc(b_base + n0 * 128 + k * 32),
                                     idesc_bf16(128, nn), (kb > 0 || k > 0) ? 1u : 0u);
                        }
                    }
                    mma_commit(wp.free_[s]);
                    wp.pend[s] = true;
                    // block kb+1 goes to the other stage once the MMAs of kb-1 are done
                    if (kb >= 1 && kb + 1 < L.nkb) {
                        ok = load_stage(wp, &maps.m[l], L, kb + 1, sW, prm.err);
                        if (!ok) break;
                    }
                }
                mma_commit(bar_done);
            }
            const bool mine = mbar_wait(bar_done, ph_done, prm.err, 4);
            ph_done ^= 1;
            if (!__syncthreads_and(ok && mine)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const bool last = (l == prm.n_layers - 1);
            // the stages are idle now: fetch the next layer's first blocks during the epilogue
            if (tid == 0) {
                const int nl = last ? 0 : l + 1;
                const bool more = !last || tile + gridDim.x < ntiles;
                if (more)
                    for (int kb = 0; kb < min(2, prm.L[nl].nkb) && ok; ++kb)
                        ok = load_stage(wp, &maps.m[nl], prm.L[nl], kb, sW, prm.err);
            }
            // ---- epilogue: TMEM -> registers (thread = point) -> bias/activation ----
            const int r = quarter * 32 + lane;
            if (!last) {
                const int Knext = prm.L[l + 1].Kpad;
                // this warp's 32-column chunks c0 = half*32 + 64 j; the TMEM read of
                // chunk j+1 is in flight while chunk j is converted
                auto store_chunk = [&](const uint32_t (&rr)[32], int c0) {
                    float x[32];
                    bias_act32(rr, x, c0, L, prm.slope);
                    unsigned char* blk = sH + (c0 / kKBlk) * (128 * 128);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint4 w4;
                        w4.x = pack_bf16(x[8 * q + 0], x[8 * q + 1]);
                        w4.y = pack_bf16(x[8 * q + 2], x[8 * q + 3]);
                        w4.z = pack_bf16(x[8 * q + 4], x[8 * q + 5]);
                        w4.w = pack_bf16(x[8 * q + 6], x[8 * q + 7]);
                        *reinterpret_cast<uint4*>(blk + swz(r, c0 % kKBlk + 8 * q)) = w4;
                    }
                };
                const int nch = (Knext - half * 32 + 63) / 64;
                uint32_t ra[32], rb[32];
                if (nch > 0) {
                    tmem_issue32(trow + (uint32_t)(half * 32), ra);
                    tmem_wait(ra);
                }
                for (int j = 0; j < nch; j += 2) {
                    const int c0 = half * 32 + 64 * j;
                    if (j + 1 < nch) tmem_issue32(trow + (uint32_t)(c0 + 64), rb);
                    store_chunk(ra, c0);
                    if (j + 1 < nch) {
                        tmem_wait(rb);
                        if (j + 2 < nch) tmem_issue32(trow + (uint32_t)(c0 + 128), ra);
                        store_chunk(rb, c0 + 64);
                        if (j + 2 < nch) tmem_wait(ra);
                    }
                }
                fence_proxy_async();
                tc_fence_before();
                __syncthreads();
                tc_fence_after();
            } else {
                // output: BF16 rows staged in the activation buffer (its MMAs are
                // done), row stride padded by 16 bytes against bank conflicts
                __nv_bfloat16* so = reinterpret_cast<__nv_bfloat16*>(sH);
                const int ldc = (NE + 31) & ~31;
                const int ldo = ldc + 8;
                for (int c0 = half * 32; c0 < ldc; c0 += 64) {
                    uint32_t rr[32];
                    tmem_issue32(trow + (uint32_t)c0, rr);
                    tmem_wait(rr);
                    float x[32];
                    bias_act32(rr, x, c0, L, prm.slope);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint4 w4;
                        w4.x = pack_bf16(x[8 * q + 0], x[8 * q + 1]);
                        w4.y = pack_bf16(x[8 * q + 2], x[8 * q + 3]);
                        w4.z = pack_bf16(x[8 * q + 4], x[8 * q + 5]);
                        w4.w = pack_bf16(x[8 * q + 6], x[8 * q + 7]);
                        *reinterpret_cast<uint4*>(so + r * ldo + c0 + 8 * q) = w4;
                    }
                }
                tc_fence_before();
                __syncthreads();
                __nv_bfloat16* dst = prm.ldos + row0 * NE;
                if ((NE & 1) == 0) {
                    const int hw = NE / 2;
                    for (int idx = tid; idx < nrows * hw; idx += kMlpThreads) {
                        const int rr = idx / hw, c2 = idx - rr * hw;
                        reinterpret_cast<uint32_t*>(dst)[idx] = *reinterpret_cast<const uint32_t*>(so + rr * ldo + 2 * c2);
                    }
                } else {
                    for (int idx = tid; idx < nrows * NE; idx += kMlpThreads) {
                        const int rr = idx / NE, c = idx - rr * NE;
                        dst[idx] = so[rr * ldo + c];
                    }
                }
                if (prm.cta_dos) {
                    for (int c = tid; c < NE; c += kMlpThreads) {
                        float sum = 0.f;
                        for (int rr = 0; rr < nrows; ++rr) sum += __bfloat162float(so[rr * ldo + c]);
                        sDos[c] += (double)sum;
                    }
                }
                __syncthreads();  // the staging buffer is the next tile's input buffer
            }
        }
        if (!ok) break;
    }
    if (prm.cta_dos)
        for (int c = tid; c < NE; c += kMlpThreads) prm.cta_dos[(int64_t)blockIdx.x * NE + c] = sDos[c];
    // after an error: let copies still in flight land before the CTA exits
    if (tid == 0)
        for (int s2 = 0; s2 < 2; ++s2)
            if (wp.inflight[s2]) wait_full(wp, s2, prm.err);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

// ---- FP64 path: plain tiled GEMM + bias + activation per layer -------------

constexpr int kT64 = 32;

__global__ void k_mlp_f64_layer(const double* __restrict__ X, int ldx, int K, const double* __restrict__ W,
                                const double* __restrict__ bias, int N, int64_t P, double slope, int act,
                                const double* __restrict__ shift, const double* __restrict__ scale,
                                double* __restrict__ Y) {
    __shared__ double sx[kT64][kT64 + 1];
    __shared__ double sw[kT64][kT64 + 1];
    const int tx = threadIdx.x % kT64, ty = threadIdx.x / kT64;  // 32 x 8 threads
    const int64_t r0 = (int64_t)blockIdx.x * kT64;
    const int n0 = blockIdx.y * kT64;
    double acc[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < K; k0 += kT64) {
        for (int i = ty; i < kT64; i += 8) {
            const int64_t r = r0 + i;
            const int k = k0 + tx;
            double v = 0.0;
            if (r < P && k < K) {
                v = X[r * ldx + k];
                if (shift) v = (v - shift[k]) * scale[k];
            }
            sx[i][tx] = v;
            const int n = n0 + i;
            sw[i][tx] = (n < N && k < K) ? W[(int64_t)n * K + k] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kT64; ++kk) {
            const double wv = sw[tx][kk];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] += sx[ty + 8 * j][kk] * wv;
        }
        __syncthreads();
    }
    const int n = n0 + tx;
    if (n >= N) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t r = r0 + ty + 8 * j;
        if (r >= P) continue;
        double v = acc[j] + bias[n];
        if (act) v = v > 0.0 ? v : slope * v;
        Y[r * N + n] = v;
    }
}

// column sums of the FP64 LDOS per block of rows
__global__ void k_colsum_f64(const double* __restrict__ L, int64_t P, int NE, int64_t rows_per_block,
                             double* __restrict__ part) {
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(P, r0 + rows_per_block);
    for (int c = threadIdx.x; c < NE; c += blockDim.x) {
        double s = 0.0;
        for (int64_t r = r0; r < r1; ++r) s += L[r * NE + c];
        part[(int64_t)blockIdx.x * NE + c] = s;
    }
}

// deterministic sum of partial rows: out[c] = sum_t part[t][c] in order of t
__global__ void k_dos_reduce(const double* __restrict__ part, int64_t nt, int NE, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= NE) return;
    double s = 0.0;
    for (int64_t t = 0; t < nt; ++t) s += part[t * NE + c];
    out[c] = s;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int pad_to(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

// ---- model upload -----------------------------------------------------------

int model_upload(Ctx* c, const mala_mlp_desc* d, Model* m) {
    m->ctx = c;
    m->n_layers = d->n_layers;
    m->dims.assign(d->dims, d->dims + d->n_layers + 1);
    m->leaky_slope = (float)d->leaky_slope;
    m->slope_d = d->leaky_slope;
    m->activate_output = d->activate_output;
    const int nl = d->n_layers;
    // MIXED layout: K padded to 64 (128-byte swizzle blocks), N padded to 16
    m->Kpad.resize(nl);
    m->Npad.resize(nl);
    m->mixed_ok = true;
    for (int l = 0; l < nl; ++l) {
        m->Kpad[l] = pad_to(m->dims[l], kKBlk);
        m->Npad[l] = pad_to(m->dims[l + 1], 16);
        if (l > 0 && m->Kpad[l] > kMaxHiddenPad) m->mixed_ok = false;
        if (m->Kpad[l] > kMaxHiddenPad || m->Npad[l] > kMaxNPad) m->mixed_ok = false;
        if (l + 1 < nl && pad_to(m->dims[l + 1], kKBlk) > kMaxHiddenPad) m->mixed_ok = false;
    }
    if (nl > kMaxLayers) m->mixed_ok = false;
    if (m->dims[nl] > 256) m->mixed_ok = false;
    auto dalloc = [&](size_t bytes, void** p) -> int {
        Ctx* r = c->root();
        if (!budget_claim(r, bytes)) return fail(MALA_ERR_OOM, "model exceeds the HBM budget");
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            r->used -= bytes;
            return fail(MALA_ERR_OOM, "cudaMalloc for the model failed");
        }
        m->bytes += bytes;
        m->allocs.push_back(*p);
        return MALA_OK;
    };
    for (int l = 0; l < nl; ++l) {
        const int K = m->dims[l], N = m->dims[l + 1];
        // FP64 copies
        void* pw = nullptr;
        void* pb = nullptr;
        MALA_TRY(dalloc(sizeof(double) * (size_t)K * N, &pw));
        MALA_TRY(dalloc(sizeof(double) * (size_t)N, &pb));
        MALA_CUDA_TRY(cudaMemcpy(pw, d->W[l], sizeof(double) * (size_t)K * N, cudaMemcpyHostToDevice));
        MALA_CUDA_TRY(cudaMemcpy(pb, d->b[l], sizeof(double) * (size_t)N, cudaMemcpyHostToDevice));
        m->Wd.push_back((double*)pw);
        m->bd.push_back((double*)pb);
        if (!m->mixed_ok) continue;
        // BF16 [Npad][Kpad], FP32 bias [Npad]
        const int Kp = m->Kpad[l], Np = m->Npad[l];
        std::vector<__nv_bfloat16> w((size_t)Np * Kp, __float2bfloat16(0.f));
        std::vector<float> bb(Np, 0.f);
        for (int n = 0; n < N; ++n) {
            for (int k = 0; k < K; ++k) w[(size_t)n * Kp + k] = __float2bfloat16((float)d->W[l][(size_t)n * K + k]);
            bb[n] = (float)d->b[l][n];
        }
        void* pwb = nullptr;
        void* pbb = nullptr;
        MALA_TRY(dalloc(sizeof(__nv_bfloat16) * w.size(), &pwb));
        MALA_TRY(dalloc(sizeof(float) * bb.size(), &pbb));
        MALA_CUDA_TRY(cudaMemcpy(pwb, w.data(), sizeof(__nv_bfloat16) * w.size(), cudaMemcpyHostToDevice));
        MALA_CUDA_TRY(cudaMemcpy(pbb, bb.data(), sizeof(float) * bb.size(), cudaMemcpyHostToDevice));
        m->Wbf.push_back(pwb);
        m->bias.push_back((float*)pbb);
    }
    // input standardisation (identity when absent)
    const int n0 = m->dims[0];
    std::vector<double> sh(n0, 0.0), sc(n0, 1.0);
    if (d->in_shift) for (int k = 0; k < n0; ++k) sh[k] = d->in_shift[k];
    if (d->in_scale) for (int k = 0; k < n0; ++k) sc[k] = d->in_scale[k];
    std::vector<float> shf(sh.begin(), sh.end()), scf(sc.begin(), sc.end());
    void* p1 = nullptr;
    void* p2 = nullptr;
    void* p3 = nullptr;
    void* p4 = nullptr;
    MALA_TRY(dalloc(sizeof(float) * n0, &p1));
    MALA_TRY(dalloc(sizeof(float) * n0, &p2));
    MALA_TRY(dalloc(sizeof(double) * n0, &p3));
    MALA_TRY(dalloc(sizeof(double) * n0, &p4));
    MALA_CUDA_TRY(cudaMemcpy(p1, shf.data(), sizeof(float) * n0, cudaMemcpyHostToDevice));
    MALA_CUDA_TRY(cudaMemcpy(p2, scf.data(), sizeof(float) * n0, cudaMemcpyHostToDevice));
    MALA_CUDA_TRY(cudaMemcpy(p3, sh.data(), sizeof(double) * n0, cudaMemcpyHostToDevice));
    MALA_CUDA_TRY(cudaMemcpy(p4, sc.data(), sizeof(double) * n0, cudaMemcpyHostToDevice));
    m->in_shift = (float*)p1;
    m->in_scale = (float*)p2;
    m->in_shift_d = (double*)p3;
    m->in_scale_d = (double*)p4;
    // tensor maps of the BF16 weights
    if (m->mixed_ok) {
        auto enc = get_encode();
        if (!enc) return fail(MALA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        for (int l = 0; l < nl; ++l) {
            const int Kp = m->Kpad[l], Np = m->Npad[l];
            int boxN = Np;
            while (boxN > 256) boxN /= 2;  // 400 -> 200
            boxN = pad_to(boxN, 8);
            while (Np % boxN) boxN -= 8;
            m->boxN.push_back(boxN);
            CUtensorMap map;
            cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Np};
            cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
            cuuint32_t box[2] = {(cuuint32_t)kKBlk, (cuuint32_t)boxN};
            cuuint32_t es[2] = {1, 1};
            CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, m->Wbf[l], dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(MALA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for layer %d", (int)r, l);
            m->maps.push_back(map);
        }
    }
    return MALA_OK;
}

void model_free(Model* m) {
    if (!m->ctx) return;
    for (void* p : m->allocs) cudaFree(p);
    m->ctx->root()->used -= m->bytes;
    m->allocs.clear();
    m->bytes = 0;
}

// ---- forward ------------------------------------------------------------------

int mlp_forward(Ctx* c, const Model* m, const void* B, int64_t P, void* ldos, double* dos_sum, mala_precision prec,
                cudaStream_t st) {
    const int nl = m->n_layers;
    const int NE = m->dims[nl];
    if (P <= 0) {
        if (dos_sum) MALA_CUDA_TRY(cudaMemsetAsync(dos_sum, 0, sizeof(double) * NE, st));
        return MALA_OK;
    }
    if (prec == MALA_MIXED) {
        if (!m->mixed_ok)
            return fail(MALA_ERR_UNSUPPORTED, "network shape outside the tensor-core kernel's limits "
                                              "(<= %d layers, hidden width <= %d, output <= 256)", kMaxLayers, kMaxHiddenPad);
        const int64_t ntiles = (P + 127) / 128;
        int dev = 0, nsm = 0;
        MALA_CUDA_TRY(cudaGetDevice(&dev));
        MALA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int grid = (int)std::min<int64_t>(ntiles, std::max(1, nsm));
        double* cta_dos = nullptr;
        if (dos_sum) {
            MALA_TRY(c->ws_tile_dos.reserve(c, sizeof(double) * (size_t)grid * NE));
            cta_dos = c->ws_tile_dos.as<double>();
        }
        TMaps maps;
        memset(&maps, 0, sizeof(maps));
        MlpParams prm;
        memset(&prm, 0, sizeof(prm));
        prm.n_layers = nl;
        for (int l = 0; l < nl; ++l) {
            maps.m[l] = m->maps[l];
            LayerDev& L = prm.L[l];
            L.K = m->dims[l];
            L.Kpad = m->Kpad[l];
            L.N = m->dims[l + 1];
            L.Npad = m->Npad[l];
            L.nkb = L.Kpad / kKBlk;
            L.boxN = m->boxN[l];
            L.act = (l < nl - 1) || m->activate_output;
            L.bias = m->bias[l];
        }
        // hidden layers feed the next layer with K = Npad rounded to 64
        for (int l = 0; l + 1 < nl; ++l) prm.L[l + 1].Kpad = pad_to(m->dims[l + 1], kKBlk), prm.L[l + 1].nkb = prm.L[l + 1].Kpad / kKBlk;
        prm.slope = m->leaky_slope;
        prm.nB = m->dims[0];
        prm.B = static_cast<const float*>(B);
        prm.shift = m->in_shift;
        prm.scale = m->in_scale;
        prm.ldos = static_cast<__nv_bfloat16*>(ldos);
        prm.cta_dos = cta_dos;
        prm.P = P;
        prm.err = c->tables.err_d + 1;
        cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        MALA_PROF(c, "k_mlp", st, (k_mlp_tc<<<(unsigned)grid, kMlpThreads, kSmemBytes, st>>>(maps, prm)));
        MALA_CUDA_TRY(cudaGetLastError());
        if (dos_sum)
            MALA_PROF(c, "k_dos_reduce", st,
                      (k_dos_reduce<<<(NE + 127) / 128, 128, 0, st>>>(cta_dos, grid, NE, dos_sum)));
        MALA_CUDA_TRY(cudaGetLastError());
        return MALA_OK;
    }
    // FP64: layer by layer through a ping-pong workspace
    int wmax = 0;
    for (int l = 1; l < nl; ++l) wmax = std::max(wmax, m->dims[l]);
    MALA_TRY(c->ws_mlp64.reserve(c, sizeof(double) * (size_t)P * (size_t)std::max(1, wmax) * 2));
    double* buf[2] = {c->ws_mlp64.as<double>(), c->ws_mlp64.as<double>() + (size_t)P * std::max(1, wmax)};
    const double* x = static_cast<const double*>(B);
    int ldx = m->dims[0];
    for (int l = 0; l < nl; ++l) {
        const int K = m->dims[l], N = m->dims[l + 1];
        double* y = (l == nl - 1) ? static_cast<double*>(ldos) : buf[l & 1];
        dim3 grid((unsigned)((P + kT64 - 1) / kT64), (unsigned)((N + kT64 - 1) / kT64));
        const int act = (l < nl - 1) || m->activate_output;
        MALA_PROF(c, "k_mlp", st,
                  (k_mlp_f64_layer<<<grid, kT64 * 8, 0, st>>>(x, ldx, K, m->Wd[l], m->bd[l], N, P, m->slope_d, act,
                                                            l == 0 ? m->in_shift_d : nullptr,
                                                            l == 0 ? m->in_scale_d : nullptr, y)));
        x = y;
        ldx = N;
    }
    MALA_CUDA_TRY(cudaGetLastError());
    if (dos_sum) {
        const int64_t rpb = 1024;
        const int64_t nb = (P + rpb - 1) / rpb;
        MALA_TRY(c->ws_tile_dos.reserve(c, sizeof(double) * (size_t)nb * NE));
        MALA_PROF(c, "k_colsum", st,
                  (k_colsum_f64<<<(unsigned)nb, 128, 0, st>>>(static_cast<const double*>(ldos), P, NE, rpb,
                                                               c->ws_tile_dos.as<double>())));
        MALA_PROF(c, "k_dos_reduce", st,
                  (k_dos_reduce<<<(NE + 127) / 128, 128, 0, st>>>(c->ws_tile_dos.as<double>(), nb, NE, dos_sum)));
        MALA_CUDA_TRY(cudaGetLastError());
    }
    return MALA_OK;
}

}  // namespace mala
