// snap_nbr.cu -- staging of a snapshot and the per-tile neighbour search.
//
// Step a1/a2 of the hot path (paper Sec. "Bispectrum descriptors",
// Eq. ionicdensity): the density around a grid point r sums over the atoms with
// |R_a - r| < R_cut, periodic images included.
//
//  * k_stage_atoms: wrap positions into the cell (x - L floor(x/L), plain
//    IEEE FP64) and drop each atom into a uniform bin (counting sort).
//  * k_neighbors: one warp per 4x4x2 tile of grid points (lane = point).  The
//    warp gathers candidate (atom, image) pairs from the bins overlapping the
//    tile's box grown by R_cut (ballot compaction into shared memory), then
//    every lane tests the candidates against its own point: FP32 outside a
//    guard band |d^2 - R_cut^2| < 1e-4 R_cut^2, and inside it the exact FP64
//    expression ((x_a + s L) - r)^2 summed as (dx^2 + dy^2) + dz^2 with no
//    fused multiply-add, so membership agrees bit for bit with that definition.
//    Positions relative to the tile origin are carried as unevaluated float
//    pairs (hi + lo, error-free sums), so the offsets fed to the FP32
//    Cayley-Klein map are as accurate as a rounded FP64 difference without
//    using the (slow) FP64 pipe per neighbour.
//    Accepted neighbours are written as Cayley-Klein parameters (a, b) and the
//    weight w_eta f_c(r) in [tile][k][lane] layout for the U-matrix kernel.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "mala_internal.h"
#include "snap_common.cuh"

namespace mala {

namespace {

// ---- FP64 helpers that forbid contraction -------------------------------

__device__ __forceinline__ double wrap_coord(double x, double L) {
    double q = __ddiv_rn(x, L);
    double fl = floor(q);
    double t = __dmul_rn(L, fl);
    return __dsub_rn(x, t);
}

__device__ __forceinline__ double grid_coord(int i, int n, double L) {
    double f = __ddiv_rn((double)i, (double)n);
    return __dmul_rn(f, L);
}

__global__ void k_stage_atoms(int n, const double* __restrict__ pos, const int* __restrict__ species,
                              const double* __restrict__ wsp_tab, int nspecies, SnapGeom g,
                              double* __restrict__ wpos, float* __restrict__ wposf, double* __restrict__ wsp,
                              int* __restrict__ bin_of, int* __restrict__ bin_count, int* __restrict__ err) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    int bc[3];
    for (int d = 0; d < 3; ++d) {
        double x = pos[3 * a + d];
        if (g.periodic[d]) x = wrap_coord(x, g.L[d]);
        wpos[(size_t)d * n + a] = x;
        const float xh = (float)x;
        wposf[(size_t)d * n + a] = xh;
        wposf[(size_t)(3 + d) * n + a] = (float)(x - (double)xh);
        double q = floor(x / g.bs[d]);
        int b = (q < 0.0) ? 0 : (q >= (double)g.nb[d] ? g.nb[d] - 1 : (int)q);
        bc[d] = b;
    }
    int s = species ? species[a] : 0;
    if (s < 0 || s >= nspecies) {
        atomicExch(err, 1);
        s = 0;
    }
    wsp[a] = wsp_tab ? wsp_tab[s] : 1.0;
    int b = bc[0] + g.nb[0] * (bc[1] + g.nb[1] * bc[2]);
    bin_of[a] = b;
    atomicAdd(&bin_count[b], 1);
}

// Exclusive scan of the bin counts (single block; bins are at most 2^21).
__global__ void k_scan_bins(int nb, const int* __restrict__ cnt, int* __restrict__ start) {
    __shared__ int part[1024];
    int t = threadIdx.x;
    int per = (nb + blockDim.x - 1) / blockDim.x;
    int lo = t * per, hi = min(nb, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            int v = part[i];
            part[i] = acc;
            acc += v;
        }
        start[nb] = acc;
    }
    __syncthreads();
    int acc = part[t];
    for (int i = lo; i < hi; ++i) {
        start[i] = acc;
        acc += cnt[i];
    }
}

__global__ void k_fill_bins(int n, const int* __restrict__ bin_of, const int* __restrict__ start,
                            int* __restrict__ fill, int* __restrict__ atoms) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    int b = bin_of[a];
    int k = atomicAdd(&fill[b], 1);
    atoms[start[b] + k] = a;
}

// Insertion sort of each bin by atom index: a deterministic candidate order.
__global__ void k_sort_bins(int nbins, const int* __restrict__ start, int* __restrict__ atoms) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    int lo = start[b], hi = start[b + 1];
    for (int i = lo + 1; i < hi; ++i) {
        int v = atoms[i];
        int j = i - 1;
        while (j >= lo && atoms[j] > v) {
            atoms[j + 1] = atoms[j];
            --j;
        }
        atoms[j + 1] = v;
    }
}

// grid coordinates r_d(i) = (i / N_d) L_d of each axis, in the exact FP64 form
__global__ void k_grid_coords(SnapGeom g, double* __restrict__ gc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n0 = g.grid[0], n1 = g.grid[1], n2 = g.grid[2];
    if (i < n0) gc[i] = grid_coord(i, n0, g.L[0]);
    else if (i < n0 + n1) gc[i] = grid_coord(i - n0, n1, g.L[1]);
    else if (i < n0 + n1 + n2) gc[i] = grid_coord(i - n0 - n1, n2, g.L[2]);
}

// error-free sum: s + e == a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (a_hi + a_lo) + (b_hi + b_lo) as a float pair
__device__ __forceinline__ void pair_add(float ah, float al, float bh, float bl, float& h, float& l) {
    float s, e;
    two_sum(ah, bh, s, e);
    const float t = __fadd_rn(__fadd_rn(al, bl), e);
    h = __fadd_rn(s, t);
    l = __fsub_rn(t, __fsub_rn(h, s));
}

__device__ __forceinline__ void split_pair(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// s * L for an image shift s, equal to __dmul_rn(s, L) (exact for |s| <= 1)
__device__ __forceinline__ double shift_mul(int s, double L) {
    if (s == 0) return 0.0;
    if (s == 1) return L;
    if (s == -1) return -L;
    return __dmul_rn((double)s, L);
}

// ---- neighbour search ------------------------------------------------------

constexpr int kWarpsPerBlock = 4;
constexpr int kCand = 128;  // candidate buffer per warp (flushed when full)

struct Cand {
    float x, y, z;      // image position relative to the tile origin: high floats
    float lx, ly, lz;   // and low floats (x + lx to about 2^-48 relative)
    int atom;
    int shift;          // packed (sx+512) | (sy+512) << 10 | (sz+512) << 20
};

__device__ __forceinline__ int pack_shift(int sx, int sy, int sz) {
    return (sx + 512) | ((sy + 512) << 10) | ((sz + 512) << 20);
}
__device__ __forceinline__ void unpack_shift(int p, int& sx, int& sy, int& sz) {
    sx = (p & 1023) - 512;
    sy = ((p >> 10) & 1023) - 512;
    sz = ((p >> 20) & 1023) - 512;
}

template <class T> struct AB;
template <> struct AB<float> { using type = float4; };
template <> struct AB<double> { using type = double4; };

__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { ::sincos(x, s, c); }
__device__ __forceinline__ float cospi_t(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_t(double x) { return ::cospi(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return ::exp(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return ::sqrt(x); }

template <class T>
__device__ __forceinline__ void cayley_klein(T dx, T dy, T dz, T inv_range, T rmin0, T rfac0_pi,
                                             typename AB<T>::type& ab, T& fc) {
    T r = sqrt_t(dx * dx + dy * dy + dz * dz);
    T t = (r - rmin0) * inv_range;
    T om = rfac0_pi * t;
    T so, co;
    sincos_t(om, &so, &co);
    fc = T(0.5) * (cospi_t(t) + T(1));
    if (r > T(0)) {
        T s = so / r;
        ab.x = co;
        ab.y = -dz * s;
        ab.z = dy * s;
        ab.w = -dx * s;
    } else {
        ab.x = T(1);
        ab.y = T(0);
        ab.z = T(0);
        ab.w = T(0);
    }
}

template <class T, bool GAUSS>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_neighbors(const BatchSnap* __restrict__ batch, int nsnap, double rcut, double rfac0, double rmin0, int64_t tile0,
                int64_t ntiles, typename AB<T>::type* __restrict__ out_ab, T* __restrict__ out_cw,
                int* __restrict__ out_cnt, int kmax, int* __restrict__ dbg_atoms, int* __restrict__ dbg_shifts,
                int* __restrict__ dbg_counts, int dbg_cap, T* __restrict__ gauss, T g_inv2s2) {
    __shared__ Cand cand[kWarpsPerBlock][kCand];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tl = (int64_t)blockIdx.x * kWarpsPerBlock + warp;  // tile index within this launch
    if (tl >= ntiles) return;
    const int si = batch_find(batch, nsnap, tile0 + tl);
    const SnapDev sd = batch[si].sd;
    const int64_t tile = tile0 + tl - batch[si].tile_off;  // tile index within its snapshot
    const SnapGeom& g = sd.g;
    const int n = g.n_atoms;
    const int tx = (int)(tile % g.tiles[0]);
    const int ty = (int)((tile / g.tiles[0]) % g.tiles[1]);
    const int tz = (int)(tile / ((int64_t)g.tiles[0] * g.tiles[1]));
    const int ix = tx * kTileX + (lane % kTileX);
    const int iy = ty * kTileY + ((lane / kTileX) % kTileY);
    const int iz = tz * kTileZ + lane / (kTileX * kTileY);
    const bool valid = ix < g.grid[0] && iy < g.grid[1] && iz < g.grid[2];
    const int64_t p = valid ? (int64_t)ix + (int64_t)g.grid[0] * ((int64_t)iy + (int64_t)g.grid[1] * iz) : -1;

    // tile box (FP64) and origin, from the per-axis coordinate tables
    double lo[3], hi[3], r[3];
    {
        const int i0[3] = {tx * kTileX, ty * kTileY, tz * kTileZ};
        const int ext[3] = {kTileX, kTileY, kTileZ};
        const int ii[3] = {ix, iy, iz};
        const double* gc = sd.gcoord;
        for (int d = 0; d < 3; ++d) {
            const int last = min(i0[d] + ext[d] - 1, g.grid[d] - 1);
            lo[d] = __ldg(gc + i0[d]);
            hi[d] = __ldg(gc + last);
            r[d] = __ldg(gc + min(ii[d], g.grid[d] - 1));
            gc += g.grid[d];
        }
    }
    float prx, pry, prz, plx, ply, plz;  // point relative to the tile origin, float pairs
    split_pair(r[0] - lo[0], prx, plx);
    split_pair(r[1] - lo[1], pry, ply);
    split_pair(r[2] - lo[2], prz, plz);
    const float bx = (float)(hi[0] - lo[0]), by = (float)(hi[1] - lo[1]), bz = (float)(hi[2] - lo[2]);
    const double rc2 = __dmul_rn(rcut, rcut);
    const float rc2f = (float)rc2;
    const float band_lo = rc2f * (1.0f - 1e-4f), band_hi = rc2f * (1.0f + 1e-4f);
    const float pre = (float)(rcut + 1e-3);
    const float pre2 = pre * pre;

    int ib_lo[3], ib_hi[3];
    for (int d = 0; d < 3; ++d) {
        // a superset of the bins that can hold a neighbour: the margin covers
        // the rounding of the reciprocal against the binning's FP64 division
        const double m = rcut + 1e-4;
        const double ibs = 1.0 / g.bs[d];
        int a = (int)floor((lo[d] - m) * ibs);
        int b = (int)floor((hi[d] + m) * ibs);
        if (!g.periodic[d]) {
            a = max(a, 0);
            b = min(b, g.nb[d] - 1);
        }
        ib_lo[d] = a;
        ib_hi[d] = b;
    }

    const T inv_range = T(1) / (T(rcut) - T(rmin0));
    const T rfac0_pi = T(rfac0 * 3.14159265358979323846);
    const T rmin0_t = T(rmin0);

    int count = 0;
    T gsum = T(0);  // Gaussian descriptor of the lane's point
    int nc = 0;     // candidates buffered
    Cand* cw = cand[warp];
    const double* wx = sd.wpos;
    const double* wy = sd.wpos + n;
    const double* wz = sd.wpos + 2 * (size_t)n;

    auto flush = [&]() {
        __syncwarp();
        for (int c = 0; c < nc; ++c) {
            const Cand cd = cw[c];
            const float dxf = cd.x - prx, dyf = cd.y - pry, dzf = cd.z - prz;
            const float d2f = __fadd_rn(__fadd_rn(__fmul_rn(dxf, dxf), __fmul_rn(dyf, dyf)), __fmul_rn(dzf, dzf));
            bool in = d2f < band_lo;
            bool decide64 = !in && d2f <= band_hi;
            int sx, sy, sz;
            unpack_shift(cd.shift, sx, sy, sz);
            double dx = 0, dy = 0, dz = 0;
            // the exact FP64 offsets: inside the guard band, and for every neighbour of the FP64 path
            if (valid && (decide64 || (in && sizeof(T) == 8))) {
                const double ux = __dadd_rn(wx[cd.atom], shift_mul(sx, g.L[0]));
                const double uy = __dadd_rn(wy[cd.atom], shift_mul(sy, g.L[1]));
                const double uz = __dadd_rn(wz[cd.atom], shift_mul(sz, g.L[2]));
                dx = __dsub_rn(ux, r[0]);
                dy = __dsub_rn(uy, r[1]);
                dz = __dsub_rn(uz, r[2]);
                if (decide64) {
                    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    in = d2 < rc2;
                }
            }
            if (valid && in) {
                if (GAUSS || count < kmax) {
                    typename AB<T>::type ab;
                    T fc;
                    T ex, ey, ez;
                    if constexpr (sizeof(T) == 8) {
                        ex = dx;
                        ey = dy;
                        ez = dz;
                    } else {
                        // (candidate - point) from the float pairs, rounded once at the end
                        float h, l;
                        pair_add(cd.x, cd.lx, -prx, -plx, h, l);
                        ex = h;
                        pair_add(cd.y, cd.ly, -pry, -ply, h, l);
                        ey = h;
                        pair_add(cd.z, cd.lz, -prz, -plz, h, l);
                        ez = h;
                    }
                    if constexpr (GAUSS) {
                        gsum += exp_t(-(ex * ex + ey * ey + ez * ez) * g_inv2s2);
                    } else {
                        cayley_klein<T>(ex, ey, ez, inv_range, rmin0_t, rfac0_pi, ab, fc);
                        const size_t o = ((size_t)tl * kmax + count) * 32 + lane;
                        out_ab[o] = ab;
                        out_cw[o] = (T)sd.wsp[cd.atom] * fc;
                    }
                }
                if (dbg_atoms && count < dbg_cap) {
                    dbg_atoms[(size_t)p * dbg_cap + count] = cd.atom;
                    int* sh = dbg_shifts + ((size_t)p * dbg_cap + count) * 3;
                    sh[0] = sx;
                    sh[1] = sy;
                    sh[2] = sz;
                }
                ++count;
            }
        }
        __syncwarp();
        nc = 0;
    };

    // image offset minus tile origin per axis, as float pairs, refreshed when the shift changes
    const float* fxh = sd.wposf;
    const float* fyh = sd.wposf + n;
    const float* fzh = sd.wposf + 2 * (size_t)n;
    const float* fxl = sd.wposf + 3 * (size_t)n;
    const float* fyl = sd.wposf + 4 * (size_t)n;
    const float* fzl = sd.wposf + 5 * (size_t)n;
    // (the shifts take one to three values per axis: each pair is formed when its shift changes)
    int sz_prev = INT_MIN, sy_prev = INT_MIN, sx_prev = INT_MIN;
    float ozh = 0.f, ozl = 0.f, oyh = 0.f, oyl = 0.f, oxh = 0.f, oxl = 0.f;
    for (int bz_ = ib_lo[2]; bz_ <= ib_hi[2]; ++bz_) {
        const int jz = ((bz_ % g.nb[2]) + g.nb[2]) % g.nb[2];
        const int sz = (bz_ - jz) / g.nb[2];
        if (sz != sz_prev) {
            split_pair(shift_mul(sz, g.L[2]) - lo[2], ozh, ozl);
            sz_prev = sz;
        }
        for (int by_ = ib_lo[1]; by_ <= ib_hi[1]; ++by_) {
            const int jy = ((by_ % g.nb[1]) + g.nb[1]) % g.nb[1];
            const int sy = (by_ - jy) / g.nb[1];
            if (sy != sy_prev) {
                split_pair(shift_mul(sy, g.L[1]) - lo[1], oyh, oyl);
                sy_prev = sy;
            }
            for (int bx_ = ib_lo[0]; bx_ <= ib_hi[0]; ++bx_) {
                const int jx = ((bx_ % g.nb[0]) + g.nb[0]) % g.nb[0];
                const int sx = (bx_ - jx) / g.nb[0];
                const int b = jx + g.nb[0] * (jy + g.nb[1] * jz);
                const int st = sd.bin_start[b], cnt = sd.bin_start[b + 1] - st;
                if (cnt == 0) continue;
                if (sx != sx_prev) {
                    split_pair(shift_mul(sx, g.L[0]) - lo[0], oxh, oxl);
                    sx_prev = sx;
                }
                for (int q0 = 0; q0 < cnt; q0 += 32) {
                    const int q = q0 + lane;
                    bool keep = false;
                    Cand cd;
                    if (q < cnt) {
                        const int a = sd.bin_atoms[st + q];
                        pair_add(__ldg(fxh + a), __ldg(fxl + a), oxh, oxl, cd.x, cd.lx);
                        pair_add(__ldg(fyh + a), __ldg(fyl + a), oyh, oyl, cd.y, cd.ly);
                        pair_add(__ldg(fzh + a), __ldg(fzl + a), ozh, ozl, cd.z, cd.lz);
                        cd.atom = a;
                        cd.shift = pack_shift(sx, sy, sz);
                        // distance from the image to the tile box
                        const float ex = fmaxf(fmaxf(-cd.x, cd.x - bx), 0.f);
                        const float ey = fmaxf(fmaxf(-cd.y, cd.y - by), 0.f);
                        const float ez = fmaxf(fmaxf(-cd.z, cd.z - bz), 0.f);
                        keep = ex * ex + ey * ey + ez * ez <= pre2;
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    const int npush = __popc(m);
                    if (nc + npush > kCand) flush();
                    if (keep) cw[nc + __popc(m & ((1u << lane) - 1u))] = cd;
                    nc += npush;
                }
            }
        }
    }
    flush();
    if constexpr (GAUSS)
        if (valid) gauss[batch[si].row_off + p] = gsum;
    if (valid && dbg_counts) dbg_counts[p] = count;
    out_cnt[tl * 32 + lane] = valid ? min(count, kmax) : 0;
    const int wmax = __reduce_max_sync(0xffffffffu, valid ? count : 0);
    if (lane == 0) atomicMax(sd.maxcnt, wmax);
}

}  // namespace

namespace {

// geometry of a snapshot and the byte offsets of its staging workspace
struct StageLayout {
    size_t o_pos, o_wpos, o_wposf, o_sp, o_wsp, o_binof, o_batoms, o_bstart, o_bcount, o_bfill, o_max, o_wtab, o_gc;
    size_t bytes;
    int ngc, ns;
};

StageLayout stage_layout(const mala_snapshot* snap, const mala_bispectrum_params* bp, double rcut, SnapGeom& g) {
    StageLayout lay{};
    g.n_atoms = snap->n_atoms;
    for (int d = 0; d < 3; ++d) {
        g.L[d] = snap->cell[d][d];
        g.periodic[d] = snap->periodic[d] ? 1 : 0;
        g.grid[d] = snap->grid[d];
        const int ext = d == 0 ? kTileX : (d == 1 ? kTileY : kTileZ);
        g.tiles[d] = (g.grid[d] + ext - 1) / ext;
        int nb = (int)floor(g.L[d] / (0.5 * rcut));
        nb = nb < 1 ? 1 : (nb > 128 ? 128 : nb);
        g.nb[d] = nb;
        g.bs[d] = g.L[d] / nb;
    }
    g.P = (int64_t)g.grid[0] * g.grid[1] * g.grid[2];
    g.n_tiles = (int64_t)g.tiles[0] * g.tiles[1] * g.tiles[2];
    g.n_bins = g.nb[0] * g.nb[1] * g.nb[2];
    const int n = g.n_atoms;
    const int nbins = g.n_bins;
    const int ns = bp && bp->n_species > 0 ? bp->n_species : 1;
    // layout of the atoms workspace
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    lay.o_pos = take(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    lay.o_wpos = take(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    lay.o_wposf = take(sizeof(float) * 6 * (size_t)(n > 0 ? n : 1));
    lay.o_sp = take(sizeof(int) * (size_t)(n > 0 ? n : 1));
    lay.o_wsp = take(sizeof(double) * (size_t)(n > 0 ? n : 1));
    lay.o_binof = take(sizeof(int) * (size_t)(n > 0 ? n : 1));
    lay.o_batoms = take(sizeof(int) * (size_t)(n > 0 ? n : 1));
    lay.o_bstart = take(sizeof(int) * (size_t)(nbins + 1));
    lay.o_bcount = take(sizeof(int) * (size_t)nbins);
    lay.o_bfill = take(sizeof(int) * (size_t)nbins);
    lay.o_max = take(sizeof(int) * 4);
    lay.o_wtab = take(sizeof(double) * (size_t)ns);
    lay.ngc = g.grid[0] + g.grid[1] + g.grid[2];
    const int ngc = lay.ngc;
    lay.o_gc = take(sizeof(double) * (size_t)(ngc > 0 ? ngc : 1));
    lay.bytes = off;
    lay.ns = ns;
    return lay;
}

}  // namespace

size_t snapshot_ws_bytes(const mala_snapshot* snap, const mala_bispectrum_params* bp, double rcut) {
    SnapGeom g{};
    return stage_layout(snap, bp, rcut, g).bytes;
}

int stage_snapshot_at(const mala_snapshot* snap, const mala_bispectrum_params* bp, double rcut, SnapDev* sd,
                      char* base, Ctx* c, cudaStream_t st) {
    SnapGeom& g = sd->g;
    const StageLayout lay = stage_layout(snap, bp, rcut, g);
    const int n = g.n_atoms;
    const int nbins = g.n_bins;
    const int ns = lay.ns;
    const int ngc = lay.ngc;
    const size_t o_pos = lay.o_pos, o_wpos = lay.o_wpos, o_wposf = lay.o_wposf, o_sp = lay.o_sp, o_wsp = lay.o_wsp,
                 o_binof = lay.o_binof, o_batoms = lay.o_batoms, o_bstart = lay.o_bstart, o_bcount = lay.o_bcount,
                 o_bfill = lay.o_bfill, o_max = lay.o_max, o_wtab = lay.o_wtab, o_gc = lay.o_gc;

    double* pos_d = (double*)(base + o_pos);
    sd->wpos = (double*)(base + o_wpos);
    sd->wposf = (float*)(base + o_wposf);
    int* sp_d = (int*)(base + o_sp);
    sd->wsp = (double*)(base + o_wsp);
    sd->bin_of = (int*)(base + o_binof);
    sd->bin_atoms = (int*)(base + o_batoms);
    sd->bin_start = (int*)(base + o_bstart);
    int* bcount = (int*)(base + o_bcount);
    sd->bin_fill = (int*)(base + o_bfill);
    sd->maxcnt = (int*)(base + o_max);
    double* wtab = (double*)(base + o_wtab);
    sd->gcoord = (double*)(base + o_gc);

    if (n > 0) {
        MALA_CUDA_TRY(cudaMemcpyAsync(pos_d, snap->pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
        if (snap->species)
            MALA_CUDA_TRY(cudaMemcpyAsync(sp_d, snap->species, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    }
    if (bp && bp->weights)
        MALA_CUDA_TRY(cudaMemcpyAsync(wtab, bp->weights, sizeof(double) * ns, cudaMemcpyHostToDevice, st));
    MALA_CUDA_TRY(cudaMemsetAsync(bcount, 0, sizeof(int) * nbins, st));
    MALA_CUDA_TRY(cudaMemsetAsync(sd->bin_fill, 0, sizeof(int) * nbins, st));
    MALA_CUDA_TRY(cudaMemsetAsync(sd->maxcnt, 0, sizeof(int) * 4, st));
    if (n > 0) {
        MALA_PROF(c, "k_stage_atoms", st,
                  (k_stage_atoms<<<(n + 127) / 128, 128, 0, st>>>(n, pos_d, snap->species ? sp_d : nullptr,
                                                                  (bp && bp->weights) ? wtab : nullptr, ns, g, sd->wpos,
                                                                  sd->wposf, sd->wsp, sd->bin_of, bcount,
                                                                  sd->maxcnt + 1)));
    }
    MALA_PROF(c, "k_scan_bins", st, (k_scan_bins<<<1, 1024, 0, st>>>(nbins, bcount, sd->bin_start)));
    if (ngc > 0) MALA_PROF(c, "k_grid_coords", st, (k_grid_coords<<<(ngc + 127) / 128, 128, 0, st>>>(g, sd->gcoord)));
    if (n > 0) {
        MALA_PROF(c, "k_fill_bins", st,
                  (k_fill_bins<<<(n + 127) / 128, 128, 0, st>>>(n, sd->bin_of, sd->bin_start, sd->bin_fill,
                                                                sd->bin_atoms)));
        MALA_PROF(c, "k_sort_bins", st,
                  (k_sort_bins<<<(nbins + 127) / 128, 128, 0, st>>>(nbins, sd->bin_start, sd->bin_atoms)));
    }
    MALA_CUDA_TRY(cudaGetLastError());
    return MALA_OK;
}

template <class T>
static void launch_neighbors_t(const BatchSnap* bs, int nsnap, double rcut, double rfac0, double rmin0, int64_t tile0,
                               int64_t ntiles, const NbrOut& out, cudaStream_t st) {
    if (ntiles <= 0) return;
    const unsigned blocks = (unsigned)((ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
    auto kern = out.gauss ? k_neighbors<T, true> : k_neighbors<T, false>;
    kern<<<blocks, kWarpsPerBlock * 32, 0, st>>>(
        bs, nsnap, rcut, rfac0, rmin0, tile0, ntiles, reinterpret_cast<typename AB<T>::type*>(out.ab),
        reinterpret_cast<T*>(out.cw), out.cnt, out.kmax, out.dbg_atoms, out.dbg_shifts, out.dbg_counts,
        out.dbg_cap, reinterpret_cast<T*>(out.gauss), (T)out.gauss_inv2s2);
}

void launch_neighbors(const BatchSnap* bs, int nsnap, double rcut, double rfac0, double rmin0, int64_t tile0,
                      int64_t ntiles, const NbrOut& out, cudaStream_t st) {
    launch_neighbors_t<float>(bs, nsnap, rcut, rfac0, rmin0, tile0, ntiles, out, st);
}

void launch_neighbors_f64(const BatchSnap* bs, int nsnap, double rcut, double rfac0, double rmin0, int64_t tile0,
                          int64_t ntiles, const NbrOut& out, cudaStream_t st) {
    launch_neighbors_t<double>(bs, nsnap, rcut, rfac0, rmin0, tile0, ntiles, out, st);
}

}  // namespace mala
