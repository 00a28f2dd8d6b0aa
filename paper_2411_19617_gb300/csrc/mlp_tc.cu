// mlp_tc.cu -- the per-point feed-forward network (paper Eq. ffnn,
// x_{l+1} = act(W_l x_l + b_l)) on the 5th-generation tensor cores, plus the
// FP64 path.
//
// MIXED path: a persistent, warp-specialised kernel, one CTA of ten warps per
// SM, walking tiles of 128 grid points (M = 128):
//   * a producer warp streams, by TMA, the tile's standardised BF16
//     descriptors (written beforehand in a padded [P][8k] layout) into the
//     activation buffer and every layer's weights W_l[N][K] through a ring of
//     four shared-memory slots, one "chunk" (a K-block of 64 times one of at
//     most two N parts of <= 208 rows) per slot, running ahead of the MMAs
//     across layers and tiles;
//   * an MMA warp issues the tcgen05.mma chain (kind::f16, BF16 x BF16 -> FP32)
//     of each layer into one tensor-memory accumulator D[128][N] (a TMEM lane
//     per point) and releases each slot by tcgen05.commit as soon as its MMAs
//     have read it;
//   * eight epilogue warps read D with tcgen05.ld (thread = point; the two
//     warps that share a TMEM lane quarter take alternate 32-column chunks),
//     add the bias (held in shared memory), apply LeakyReLU on hidden layers
//     and write the BF16 activations back as the next layer's A operand in the
//     UMMA K-major, 128-byte-swizzled layout; the last layer's values go,
//     rounded to BF16, into a dense [128][N_E] staging tile that one bulk copy
//     stores to the LDOS, and their column sums over the tile's points (a
//     transposing butterfly across the warp, then the four lane quarters in a
//     fixed order, in FP64) go into the CTA's DOS partial; the partials of all
//     CTAs are summed in CTA order afterwards, so the DOS does not depend on
//     timing.
// The next tile's descriptors land (in the activation blocks that the staging
// tile does not use) while the last epilogue of the current tile runs.  Every
// wait is bounded (about one second of clock cycles); on expiry the kernel
// records an error code, raises a shared abort flag that ends every other
// wait, lets its copies land, frees its tensor memory and returns.
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

constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kProducerWarp = kEpiWarps;      // TMA issue
constexpr int kMmaWarp = kEpiWarps + 1;       // tcgen05.mma issue, TMEM owner
constexpr int kMlpThreads = (kEpiWarps + 2) * 32;
constexpr int kMaxLayers = 4;
constexpr int kKBlk = 64;                     // K elements per swizzle block (128 bytes of BF16)
constexpr int kHBlocks = 7;
constexpr int kMaxHiddenPad = kHBlocks * kKBlk;  // widest K of a hidden activation: 448
constexpr int kBlkBytes = 128 * 128;             // one [128 rows][64] BF16 K-block
constexpr int kHBytes = kHBlocks * kBlkBytes;    // 114688
constexpr int kRing = 4;                         // weight slots
constexpr int kChunkRows = 208;                  // rows of the widest weight chunk
constexpr int kChunkBytes = kChunkRows * 128;    // 26624
constexpr int kMaxParts = 2;
constexpr int kMaxNPad = 400;                    // widest layer output (two parts, cut at a K-block boundary)
constexpr int kMaxNE = 256;                      // widest output layer (staging tile <= 4 K-blocks)
constexpr int kMaxInBlocks = 2;                  // input K-blocks (descriptor count + 2 <= 128)
constexpr int kQOff = 4 * kBlkBytes;             // column sums of the four lane quarters, behind the staging tile
constexpr int kSmemBytes = kHBytes + kRing * kChunkBytes + kMaxNE * 8 + 256 /* barriers */ + 1024 /* alignment */;
static_assert(kSmemBytes <= 232448, "shared memory of the network kernel");
static_assert(kQOff + 4 * kMaxNE * 4 <= (kHBlocks - kMaxInBlocks) * kBlkBytes, "quarter sums overlap the input");
constexpr long long kWaitCycles = 2000000000LL;

// The bias rides in the MMA: the A operand of every layer carries two
// constant-one columns right after its K real columns, and the weights carry
// the bias there as a BF16 pair (b_hi = bf16(b), b_lo = bf16(b - b_hi)), so the
// FP32 accumulator already holds W x + b (to about 2^-16 of b).

struct LayerDev {
    int nkb;              // K-blocks of 64 (the A operand's width / 64)
    int N, Npad;          // output width, padded to 16
    int nparts;           // N parts (one commit each; part boundaries on K-block boundaries)
    int prow[kMaxParts];  // rows of each part (multiples of 16, <= kChunkRows)
    int pn0[kMaxParts];   // first output column of each part (multiples of 64)
    int act;              // apply LeakyReLU
};

struct MlpParams {
    int n_layers;
    LayerDev L[kMaxLayers];
    float slope;
    int slope_max;          // 0 <= slope <= 1: LeakyReLU as max(t, slope t)
    int nin;                // input K-blocks (layer 0's nkb)
    __nv_bfloat16* ldos;    // [P][N_E]
    int bulk_out;           // LDOS 16-byte aligned: full tiles leave by one bulk copy
    double* cta_dos;        // [gridDim.x][N_E] or nullptr
    int64_t P;
    int* err;
};

struct TMaps {
    CUtensorMap in;                          // standardised BF16 descriptors [P][nin_cols] (+ the ones columns)
    CUtensorMap w[kMaxLayers][kMaxParts];    // BF16 weights [Npad][Kpad], one map per part height
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

// Bounded wait: false if the phase did not complete in time (then *err is set
// and the abort flag raised) or if another role has raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, volatile int* abort_flag, int* err,
                                          int code) {
    const long long t0 = clock64();
    while (!mbar_try(bar, phase)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            atomicCAS(err, 0, code);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// a wait at teardown: for copies still in flight, no abort shortcut
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try(bar, phase))
        if (clock64() - t0 > kWaitCycles) return;
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
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }
// barrier of the epilogue warps that also ORs a flag over them: the same answer in every thread
__device__ __forceinline__ bool epi_sync_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kEpiThreads)
        : "memory");
    return r != 0;
}

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

// tcgen05.st of 16 registers into 16 consecutive columns of the warp's lane
// quarter, then the wait for it; and the matching 16-column read
__device__ __forceinline__ void tmem_park16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_park1(uint32_t taddr, uint32_t v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v) : "memory");
}
__device__ __forceinline__ void tmem_park_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_unpark17(uint32_t taddr, uint32_t (&r)[16], uint32_t& v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr + 16u));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                   "+r"(v)
                 :
                 : "memory");
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

// activation of 32 accumulator columns c0.. (bias already inside): columns
// beyond the layer's N become the constant-one columns of the next layer's
// bias (N and N + 1) or zero
__device__ __forceinline__ void act32(const uint32_t (&r)[32], float (&x)[32], int c0, const LayerDev& L, float slope,
                                      bool slope_max, bool ones) {
    if (c0 + 32 <= L.N) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float t = __uint_as_float(r[i]);
            if (L.act) t = slope_max ? fmaxf(t, slope * t) : (t > 0.f ? t : slope * t);
            x[i] = t;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int c = c0 + i;
            float t = __uint_as_float(r[i]);
            if (L.act) t = slope_max ? fmaxf(t, slope * t) : (t > 0.f ? t : slope * t);
            x[i] = c < L.N ? t : ((ones && (c == L.N || c == L.N + 1)) ? 1.f : 0.f);
        }
    }
}

// v: this lane's values of 32 columns; returns the sum over the warp's 32
// lanes of column `lane` (a transposing butterfly: 31 shuffles, fixed order)
__device__ __forceinline__ float warp_colsum32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// A-operand K-block kb of layer l (l > 0) is written by the part of layer
// l - 1 that holds its first column (part boundaries sit on K-block
// boundaries; the padding blocks belong to the last part)
__device__ __forceinline__ int part_of_col(const LayerDev& L, int col) {
    return (L.nparts > 1 && col >= L.pn0[1]) ? 1 : 0;
}

__global__ void __launch_bounds__(kMlpThreads, 1) k_mlp_tc(const __grid_constant__ TMaps maps, MlpParams prm) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sH = sm;                                  // activations, K-blocks of [128][64] BF16
    unsigned char* sRing = sm + kHBytes;                     // weight chunks
    double* sDos = reinterpret_cast<double*>(sRing + kRing * kChunkBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sDos + kMaxNE);
    // barriers: full[kRing] | empty[kRing] | in_full | in_free | acc[2] | epi[2]
    constexpr int B_FULL = 0, B_EMPTY = kRing, B_IN_FULL = 2 * kRing, B_IN_FREE = 2 * kRing + 1,
                  B_ACC = 2 * kRing + 2, B_EPI = 2 * kRing + 4, NBARS = 2 * kRing + 6;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + NBARS);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (prm.P + 127) / 128;
    const int nl = prm.n_layers;
    const int NE = prm.L[nl - 1].N;
    auto bar = [&](int i) { return smem_u32(&bars[i]); };

    if (tid == 0) {
        for (int i = 0; i < B_EPI; ++i) mbar_init(bar(i), 1);
        mbar_init(bar(B_EPI), kEpiWarps);
        mbar_init(bar(B_EPI + 1), kEpiWarps);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int c = tid; c < NE; c += kMlpThreads) sDos[c] = 0.0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == kProducerWarp) {
        // ---- producer: the next tiles' inputs and the weight chunks, in consumption order
        //      (per layer: part-major, K-blocks within a part) ----
        if (lane == 0) {
            for (int l = 0; l < nl; ++l)
                for (int p = 0; p < prm.L[l].nparts; ++p)
                    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.w[l][p])) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.in)) : "memory");
            uint32_t chunk = 0, in_ph = 0, issued_in = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                if (issued_in > 0) {  // the previous tile's last MMAs have read the activation buffer
                    ok = mbar_wait(bar(B_IN_FREE), in_ph, abort_flag, prm.err, 5);
                    in_ph ^= 1;
                    if (!ok) break;
                }
                mbar_expect_tx(bar(B_IN_FULL), (uint32_t)prm.nin * kBlkBytes);
                for (int kb = 0; kb < prm.nin; ++kb)
                    tma_load_2d(smem_u32(sH + (kHBlocks - prm.nin + kb) * kBlkBytes), &maps.in, kb * kKBlk,
                                (int)(tile * 128), bar(B_IN_FULL));
                ++issued_in;
                for (int l = 0; l < nl && ok; ++l) {
                    const LayerDev& L = prm.L[l];
                    for (int p = 0; p < L.nparts && ok; ++p)
                        for (int kb = 0; kb < L.nkb; ++kb, ++chunk) {
                            const uint32_t slot = chunk % kRing;
                            if (chunk >= (uint32_t)kRing) {
                                ok = mbar_wait(bar(B_EMPTY + slot), ((chunk / kRing) - 1) & 1, abort_flag, prm.err, 3);
                                if (!ok) break;
                            }
                            mbar_expect_tx(bar(B_FULL + slot), (uint32_t)L.prow[p] * 128u);
                            tma_load_2d(smem_u32(sRing + slot * kChunkBytes), &maps.w[l][p], kb * kKBlk, L.pn0[p],
                                        bar(B_FULL + slot));
                        }
                }
            }
            // let the copies still in flight land before the CTA can exit
            for (uint32_t s2 = 0; s2 < (uint32_t)kRing; ++s2) {
                if (chunk > s2) {
                    const uint32_t last = chunk - 1 - ((chunk - 1 - s2) % kRing);  // last chunk issued to slot s2
                    mbar_drain(bar(B_FULL + s2), (last / kRing) & 1);
                }
            }
            if (issued_in > 0) mbar_drain(bar(B_IN_FULL), (issued_in - 1) & 1);
        }
    } else if (warp == kMmaWarp) {
        // ---- MMA issuer: a part's K-blocks, then its commit; every A block and
        //      TMEM column waits only for the epilogue part that produces or reads it ----
        if (lane == 0) {
            uint32_t chunk = 0, in_ph = 0, epi_ph = 0;  // epi_ph: bit q = phase of epilogue barrier q
            bool ok = true, first = true;
            auto wait_epi = [&](int q) {
                ok = mbar_wait(bar(B_EPI + q), (epi_ph >> q) & 1u, abort_flag, prm.err, 4);
                epi_ph ^= 1u << q;
                tc_fence_after();
            };
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int l = 0; l < nl && ok; ++l) {
                    const LayerDev& L = prm.L[l];
                    const LayerDev& Lp = prm.L[l == 0 ? nl - 1 : l - 1];  // the layer whose epilogue comes before
                    uint32_t waited = 0;  // parts of that epilogue waited for in this layer
                    if (l == 0) {
                        ok = mbar_wait(bar(B_IN_FULL), in_ph, abort_flag, prm.err, 6);
                        in_ph ^= 1;
                        tc_fence_after();
                        // the previous tile's last epilogue must have read every accumulator column
                        if (!first)
                            for (int q = 0; q < Lp.nparts && ok; ++q) wait_epi(q);
                        waited = 3u;
                        if (!ok) break;
                    }
                    first = false;
                    const int ablk0 = (l == 0) ? kHBlocks - prm.nin : 0;
                    for (int p = 0; p < L.nparts && ok; ++p) {
                        // TMEM columns of this part: every part of the previous epilogue reading them
                        for (int q = 0; q < Lp.nparts && ok; ++q) {
                            const int q0 = Lp.pn0[q], q1 = (q + 1 < Lp.nparts) ? Lp.pn0[q + 1] : (1 << 30);
                            if (!(waited >> q & 1) && q0 < L.pn0[p] + L.prow[p] && L.pn0[p] < q1) {
                                wait_epi(q);
                                waited |= 1u << q;
                            }
                        }
                        for (int kb = 0; kb < L.nkb && ok; ++kb, ++chunk) {
                            if (l > 0) {  // the A block's producer part
                                const int q = part_of_col(Lp, kb * kKBlk);
                                if (!(waited >> q & 1)) {
                                    wait_epi(q);
                                    waited |= 1u << q;
                                    if (!ok) break;
                                }
                            }
                            const uint32_t slot = chunk % kRing;
                            ok = mbar_wait(bar(B_FULL + slot), (chunk / kRing) & 1, abort_flag, prm.err, 2);
                            if (!ok) break;
                            tc_fence_after();
                            const uint32_t a_base = smem_u32(sH + (ablk0 + kb) * kBlkBytes);
                            const uint32_t b_base = smem_u32(sRing + slot * kChunkBytes);
                            const uint32_t idesc = idesc_bf16(128, L.prow[p]);
#pragma unroll
                            for (int k = 0; k < kKBlk / 16; ++k)
                                mma_bf16(tmem + (uint32_t)L.pn0[p], sdesc(a_base + k * 32), sdesc(b_base + k * 32), idesc,
                                         (kb > 0 || k > 0) ? 1u : 0u);
                            mma_commit(bar(B_EMPTY + slot));
                        }
                        if (!ok) break;
                        mma_commit(bar(B_ACC + p));
                    }
                    if (!ok) break;
                    // every part of the previous epilogue has been waited for (all A blocks are read)
                    for (int q = 0; q < Lp.nparts && ok && l > 0; ++q)
                        if (!(waited >> q & 1)) wait_epi(q);
                    if (l == nl - 1) mma_commit(bar(B_IN_FREE));
                }
            }
        }
    } else {
        // ---- epilogue warps: TMEM -> registers (thread = point) -> activation -> shared memory ----
        const int quarter = warp & 3, half = warp >> 2;
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
        const int r = quarter * 32 + lane;
        float* sQ = reinterpret_cast<float*>(sH + kQOff);  // [4][NE] column sums of the lane quarters
        __nv_bfloat16* so = reinterpret_cast<__nv_bfloat16*>(sH);
        const bool smax = prm.slope_max != 0;
        uint32_t acc_ph = 0;  // bit p = phase of accumulator barrier p
        bool ok = true, store_pending = false;
        // one 32-column chunk c0 of this thread's row: activation, then into the next
        // layer's A block (swizzled) or, for the last layer, into the staging row with
        // the chunk's column sums over the warp's rows (returned for lane c)
        auto chunk_vals = [&](const uint32_t (&rr)[32], int c0, const LayerDev& L, bool last, int nrows,
                              uint32_t (&pk)[16], float& cs) {
            float x[32];
            act32(rr, x, c0, L, prm.slope, smax, !last);
#pragma unroll
            for (int q = 0; q < 16; ++q) pk[q] = pack_bf16(x[2 * q], x[2 * q + 1]);
            if (last && prm.cta_dos) {
                // column sums of the rounded values of the tile's real rows and columns
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk[q]));
                    x[2 * q] = (r < nrows && c0 + 2 * q < NE) ? f.x : 0.f;
                    x[2 * q + 1] = (r < nrows && c0 + 2 * q + 1 < NE) ? f.y : 0.f;
                }
                cs = warp_colsum32(x);
            }
        };
        auto chunk_store = [&](const uint32_t (&pk)[16], float cs, int c0, bool last) {
            if (!last) {
                unsigned char* blk = sH + (c0 / kKBlk) * kBlkBytes;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<uint4*>(blk + swz(r, c0 % kKBlk + 8 * q)) =
                        make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            } else {
                __nv_bfloat16* orow = so + (size_t)r * NE;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&pk[q]);
                    if (c0 + 2 * q < NE) orow[c0 + 2 * q] = h.x;
                    if (c0 + 2 * q + 1 < NE) orow[c0 + 2 * q + 1] = h.y;
                }
                if (prm.cta_dos && c0 + lane < NE) sQ[quarter * NE + c0 + lane] = cs;
            }
        };
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int64_t row0 = tile * 128;
            const int nrows = (int)min((int64_t)128, prm.P - row0);
            for (int l = 0; l < nl && ok; ++l) {
                const LayerDev& L = prm.L[l];
                const bool last = l == nl - 1;
                const int cend = last ? ((NE + 31) & ~31) : prm.L[l + 1].nkb * kKBlk;
                bool acc1_taken = false;  // the second part's accumulator barrier already waited for
                for (int p = 0; p < L.nparts; ++p) {
                    bool got = true;
                    if (!(p == 1 && acc1_taken)) {
                        got = mbar_wait(bar(B_ACC + p), (acc_ph >> p) & 1u, abort_flag, prm.err, 7);
                        acc_ph ^= 1u << p;
                        tc_fence_after();
                    }
                    // before the first writes of a tile: the previous tile's output copy has read the staging tile
                    if (l == 0 && p == 0 && tid == 0 && store_pending)
                        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    if (l == 0 && p == 0) store_pending = false;
                    // one decision for all epilogue warps (none may stop alone: they share named barriers)
                    if (epi_sync_any(!got || *abort_flag)) {
                        ok = false;
                        break;
                    }
                    const int cb = L.pn0[p];
                    const int ce = (p + 1 < L.nparts) ? L.pn0[p + 1] : cend;
                    const int nch = (ce - cb - half * 32 + 63) / 64;  // this warp's chunks: cb + half*32 + 64 j
                    // the layer's A blocks: the input blocks for layer 0, all of them afterwards
                    const bool park = p == 0 && L.nparts == 2 && (l > 0 || L.pn0[1] / kKBlk > kHBlocks - prm.nin);
                    if (park) {
                        // The second part's MMAs still read the activations this part overwrites: while
                        // they run, convert this part's chunks and park the packed results (and column
                        // sums) in the chunks' own, already read, accumulator columns; store them to
                        // shared memory once every MMA of the layer is done.
                        for (int j = 0; j < nch; ++j) {
                            const int c0 = cb + half * 32 + 64 * j;
                            uint32_t rr[32], pk[16];
                            float cs = 0.f;
                            tmem_issue32(trow + (uint32_t)c0, rr);
                            tmem_wait(rr);
                            chunk_vals(rr, c0, L, last, nrows, pk, cs);
                            tmem_park16(trow + (uint32_t)c0, pk);
                            tmem_park1(trow + (uint32_t)(c0 + 16), __float_as_uint(cs));
                        }
                        tmem_park_wait();
                        got = mbar_wait(bar(B_ACC + 1), (acc_ph >> 1) & 1u, abort_flag, prm.err, 7);
                        acc_ph ^= 2u;
                        acc1_taken = true;
                        tc_fence_after();
                        if (epi_sync_any(!got || *abort_flag)) {
                            ok = false;
                            break;
                        }
                        for (int j = 0; j < nch; ++j) {
                            const int c0 = cb + half * 32 + 64 * j;
                            uint32_t pk[16], csu;
                            tmem_unpark17(trow + (uint32_t)c0, pk, csu);
                            chunk_store(pk, __uint_as_float(csu), c0, last);
                        }
                    } else {
                        for (int j = 0; j < nch; ++j) {
                            const int c0 = cb + half * 32 + 64 * j;
                            uint32_t rr[32], pk[16];
                            float cs = 0.f;
                            tmem_issue32(trow + (uint32_t)c0, rr);
                            tmem_wait(rr);
                            chunk_vals(rr, c0, L, last, nrows, pk, cs);
                            chunk_store(pk, cs, c0, last);
                        }
                    }
                    // this part of the accumulator has been read and its outputs written
                    fence_proxy_async();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(B_EPI + p));
                }
                if (!ok) break;
                if (last) {
                    epi_sync();
                    if (prm.cta_dos && tid < NE)
                        sDos[tid] += (((double)sQ[tid] + (double)sQ[NE + tid]) + (double)sQ[2 * NE + tid]) +
                                     (double)sQ[3 * NE + tid];
                    __nv_bfloat16* dst = prm.ldos + row0 * NE;
                    if (prm.bulk_out && nrows == 128) {
                        if (tid == 0) {
                            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                                         "r"(smem_u32(so)), "r"((uint32_t)(128 * NE * 2))
                                         : "memory");
                            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                        }
                        store_pending = true;
                    } else {
                        for (int idx = tid; idx < nrows * NE; idx += kEpiThreads) dst[idx] = so[idx];
                    }
                }
            }
        }
        if (tid == 0 && store_pending) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        if (prm.cta_dos)
            for (int c = tid; c < NE; c += kEpiThreads) prm.cta_dos[(int64_t)blockIdx.x * NE + c] = sDos[c];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

// standardised BF16 copy of the descriptors for the network's input TMA:
// Bh[p][k] = (B[p][k] - shift[k]) * scale[k] for k < nB, 1 at k = nB and nB + 1
// (the bias columns), 0 up to the padded width nBh
__global__ void k_mlp_in(const float* __restrict__ B, int64_t P, int nB, int nBh, const float* __restrict__ shift,
                         const float* __restrict__ scale, __nv_bfloat16* __restrict__ Bh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one 8-column group
    const int g = nBh / 8;
    if (i >= P * g) return;
    const int64_t p = i / g;
    const int k0 = (int)(i - p * g) * 8;
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float v[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int k = k0 + 2 * j + t;
            v[t] = k < nB ? (__ldg(B + p * nB + k) - __ldg(shift + k)) * __ldg(scale + k) : (k < nB + 2 ? 1.f : 0.f);
        }
        w[j] = pack_bf16(v[0], v[1]);
    }
    *reinterpret_cast<uint4*>(Bh + p * nBh + k0) = make_uint4(w[0], w[1], w[2], w[3]);
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
    // MIXED layout: K + 2 (the two bias columns) padded to 64 (128-byte swizzle
    // blocks), N padded to 16 and cut into at most two parts of <= 208 rows at a
    // K-block boundary (one ring slot and one commit each)
    m->Kpad.resize(nl);
    m->Npad.resize(nl);
    m->nparts.assign(nl, 1);
    m->prow.assign(2 * nl, 0);
    m->pn0.assign(2 * nl, 0);
    m->mixed_ok = nl <= kMaxLayers && m->dims[nl] <= kMaxNE;
    for (int l = 0; l < nl; ++l) {
        m->Kpad[l] = pad_to(m->dims[l] + 2, kKBlk);
        m->Npad[l] = pad_to(m->dims[l + 1], 16);
        const int Np = m->Npad[l];
        if ((l == 0 && m->Kpad[l] > kMaxInBlocks * kKBlk) || m->Kpad[l] > kMaxHiddenPad || Np > kMaxNPad)
            m->mixed_ok = false;
        if (Np <= kChunkRows) {
            m->prow[2 * l] = Np;
        } else {
            const int p0 = std::max(kKBlk * ((Np - kChunkRows + kKBlk - 1) / kKBlk), kKBlk * (Np / (2 * kKBlk)));
            if (p0 > kChunkRows || Np - p0 > kChunkRows) m->mixed_ok = false;
            m->nparts[l] = 2;
            m->prow[2 * l] = p0;
            m->prow[2 * l + 1] = Np - p0;
            m->pn0[2 * l + 1] = p0;
        }
    }
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
        // BF16 [Npad][Kpad]; the bias as a BF16 pair in columns K and K + 1, which
        // meet the constant-one columns of the A operand
        const int Kp = m->Kpad[l], Np = m->Npad[l];
        std::vector<__nv_bfloat16> w((size_t)Np * Kp, __float2bfloat16(0.f));
        for (int n = 0; n < N; ++n) {
            for (int k = 0; k < K; ++k) w[(size_t)n * Kp + k] = __float2bfloat16((float)d->W[l][(size_t)n * K + k]);
            const double b = d->b[l][n];
            const __nv_bfloat16 hi = __float2bfloat16((float)b);
            w[(size_t)n * Kp + K] = hi;
            w[(size_t)n * Kp + K + 1] = __float2bfloat16((float)(b - (double)__bfloat162float(hi)));
        }
        void* pwb = nullptr;
        MALA_TRY(dalloc(sizeof(__nv_bfloat16) * w.size(), &pwb));
        MALA_CUDA_TRY(cudaMemcpy(pwb, w.data(), sizeof(__nv_bfloat16) * w.size(), cudaMemcpyHostToDevice));
        m->Wbf.push_back(pwb);
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
        m->maps.assign(2 * nl, CUtensorMap{});
        for (int l = 0; l < nl; ++l) {
            const int Kp = m->Kpad[l], Np = m->Npad[l];
            for (int p = 0; p < m->nparts[l]; ++p) {
                CUtensorMap map;
                cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Np};
                cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
                cuuint32_t box[2] = {(cuuint32_t)kKBlk, (cuuint32_t)m->prow[2 * l + p]};
                cuuint32_t es[2] = {1, 1};
                CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, m->Wbf[l], dims, strides, box, es,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS)
                    return fail(MALA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for layer %d", (int)r, l);
                m->maps[2 * l + p] = map;
            }
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

void mlp_ws_needs(Ctx* c, const Model* m, int64_t P, bool dos, mala_precision prec, WsNeeds& out) {
    const int nl = m->n_layers;
    const int NE = m->dims[nl];
    if (P <= 0) return;
    if (prec == MALA_MIXED) {
        const int64_t ntiles = (P + 127) / 128;
        const int grid = (int)std::min<int64_t>(ntiles, std::max(1, c->num_sms));
        if (dos) out.add(c->ws_tile_dos, sizeof(double) * (size_t)grid * NE);
        out.add(c->ws_mlp_in, sizeof(__nv_bfloat16) * (size_t)P * pad_to(m->dims[0] + 2, 8));
        return;
    }
    int wmax = 0;
    for (int l = 1; l < nl; ++l) wmax = std::max(wmax, m->dims[l]);
    out.add(c->ws_mlp64, sizeof(double) * (size_t)P * (size_t)std::max(1, wmax) * 2);
    if (dos) out.add(c->ws_tile_dos, sizeof(double) * (size_t)((P + 1023) / 1024) * NE);
}

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
                                              "(<= %d layers, input <= %d, hidden width <= %d, output <= %d)",
                        kMaxLayers, kMaxInBlocks * kKBlk - 2, kMaxNPad, kMaxNE);
        const int64_t ntiles = (P + 127) / 128;
        if (ntiles > (int64_t)INT32_MAX / 2) return fail(MALA_ERR_UNSUPPORTED, "too many grid points for the network");
        const int grid = (int)std::min<int64_t>(ntiles, std::max(1, c->num_sms));
        double* cta_dos = nullptr;
        if (dos_sum) {
            MALA_TRY(c->ws_tile_dos.reserve(c, sizeof(double) * (size_t)grid * NE));
            cta_dos = c->ws_tile_dos.as<double>();
        }
        // standardised BF16 input rows, padded to a multiple of 8 (16 bytes) for the input TMA
        const int nB = m->dims[0];
        const int nBh = pad_to(nB + 2, 8);  // + the two bias columns
        MALA_TRY(c->ws_mlp_in.reserve(c, sizeof(__nv_bfloat16) * (size_t)P * nBh));
        __nv_bfloat16* Bh = c->ws_mlp_in.as<__nv_bfloat16>();
        {
            const int64_t groups = P * (nBh / 8);
            MALA_PROF(c, "k_mlp_in", st,
                      (k_mlp_in<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(static_cast<const float*>(B), P, nB, nBh,
                                                                                  m->in_shift, m->in_scale, Bh)));
        }
        auto enc = get_encode();
        if (!enc) return fail(MALA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        TMaps maps;
        memset(&maps, 0, sizeof(maps));
        {
            cuuint64_t dims[2] = {(cuuint64_t)nBh, (cuuint64_t)P};
            cuuint64_t strides[1] = {(cuuint64_t)nBh * 2};
            cuuint32_t box[2] = {(cuuint32_t)kKBlk, 128u};
            cuuint32_t es[2] = {1, 1};
            CUresult r = enc(&maps.in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Bh, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(MALA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for the input", (int)r);
        }
        MlpParams prm;
        memset(&prm, 0, sizeof(prm));
        prm.n_layers = nl;
        for (int l = 0; l < nl; ++l) {
            LayerDev& L = prm.L[l];
            L.nkb = m->Kpad[l] / kKBlk;
            L.N = m->dims[l + 1];
            L.Npad = m->Npad[l];
            L.nparts = m->nparts[l];
            for (int p = 0; p < L.nparts; ++p) {
                L.prow[p] = m->prow[2 * l + p];
                L.pn0[p] = m->pn0[2 * l + p];
                maps.w[l][p] = m->maps[2 * l + p];
            }
            L.act = (l < nl - 1) || m->activate_output;
        }
        prm.slope = m->leaky_slope;
        prm.slope_max = (m->leaky_slope >= 0.f && m->leaky_slope <= 1.f) ? 1 : 0;
        prm.nin = m->Kpad[0] / kKBlk;
        prm.ldos = static_cast<__nv_bfloat16*>(ldos);
        prm.bulk_out = (reinterpret_cast<uintptr_t>(ldos) & 15) == 0;
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
