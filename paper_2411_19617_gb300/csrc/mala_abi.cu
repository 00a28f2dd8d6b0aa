// mala_abi.cu -- the C ABI declared in include/mala.h: context, error
// reporting, workspaces and the descriptor step (neighbour lists, u, B).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "mala_internal.h"
#include "snap_common.cuh"

namespace mala {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

DevBuf::~DevBuf() { release(); }

void DevBuf::release() {
    if (ptr) {
        cudaFree(ptr);
        if (owner) owner->root()->used -= bytes;
    }
    ptr = nullptr;
    bytes = 0;
}

bool budget_claim(Ctx* r, size_t n) {
    if (!r->budget) {
        r->used += n;
        return true;
    }
    size_t cur = r->used.load();
    do {
        if (cur + n > r->budget) return false;
    } while (!r->used.compare_exchange_weak(cur, cur + n));
    return true;
}

int DevBuf::reserve(Ctx* ctx, size_t n) {
    if (n <= bytes && ptr) return MALA_OK;
    Ctx* r = ctx->root();
    if (owner && owner != ctx) release();
    owner = ctx;
    const size_t old = ptr ? bytes : 0;
    // the bytes beyond the old buffer come first from what admission set aside
    // for this context, then from the budget; the old buffer's bytes carry over
    const size_t extra = n > old ? n - old : 0;
    const size_t from_held = std::min(extra, ctx->held);
    if (!budget_claim(r, extra - from_held))
        return fail(MALA_ERR_OOM, "workspace of %zu bytes exceeds the HBM budget (%zu of %zu in use)", n,
                    (size_t)r->used, r->budget);
    ctx->held -= from_held;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    if (n == 0) {
        r->used -= old;  // nothing kept: the old buffer's bytes go back
        return MALA_OK;
    }
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();
        r->used -= old + extra;
        return fail(MALA_ERR_OOM, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
    }
    bytes = n;
    if (n < old) r->used -= old - n;
    return MALA_OK;
}

// ---- validation ---------------------------------------------------------

int check_snapshot(const mala_snapshot* s) {
    if (!s) return fail(MALA_ERR_INVALID_ARG, "snapshot is NULL");
    if (s->n_atoms < 0) return fail(MALA_ERR_INVALID_ARG, "n_atoms < 0");
    if (s->n_atoms > 0 && !s->pos) return fail(MALA_ERR_INVALID_ARG, "positions are NULL");
    for (int d = 0; d < 3; ++d) {
        if (s->grid[d] < 1) return fail(MALA_ERR_INVALID_ARG, "grid[%d] = %d < 1", d, s->grid[d]);
        if (!(s->cell[d][d] > 0.0) || !std::isfinite(s->cell[d][d]))
            return fail(MALA_ERR_INVALID_ARG, "cell[%d][%d] must be positive and finite", d, d);
        for (int e = 0; e < 3; ++e)
            if (e != d && s->cell[d][e] != 0.0)
                return fail(MALA_ERR_UNSUPPORTED, "only orthorhombic (diagonal) cells are supported");
    }
    for (int64_t i = 0; i < 3 * (int64_t)s->n_atoms; ++i)
        if (!std::isfinite(s->pos[i])) return fail(MALA_ERR_INVALID_ARG, "position %lld is not finite", (long long)i / 3);
    const double P = (double)s->grid[0] * s->grid[1] * s->grid[2];
    if (P > 4.0e9) return fail(MALA_ERR_UNSUPPORTED, "grid of %.3g points is too large", P);
    return MALA_OK;
}

int check_bparams(const mala_bispectrum_params* bp) {
    if (!bp) return fail(MALA_ERR_INVALID_ARG, "bispectrum params are NULL");
    if (bp->twojmax < 0 || (bp->twojmax & 1) || bp->twojmax > kTJMax)
        return fail(MALA_ERR_UNSUPPORTED, "twojmax = %d: this build supports even values 0..%d", bp->twojmax, kTJMax);
    if (!(bp->rcut > 0.0) || !std::isfinite(bp->rcut)) return fail(MALA_ERR_INVALID_ARG, "rcut must be > 0");
    if (!(bp->rmin0 >= 0.0) || !(bp->rmin0 < bp->rcut)) return fail(MALA_ERR_INVALID_ARG, "need 0 <= rmin0 < rcut");
    if (!std::isfinite(bp->rfac0) || !std::isfinite(bp->wself)) return fail(MALA_ERR_INVALID_ARG, "rfac0/wself not finite");
    if (bp->weights && bp->n_species < 1) return fail(MALA_ERR_INVALID_ARG, "weights given with n_species < 1");
    return MALA_OK;
}

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---- descriptor step ------------------------------------------------------

// ---- tile-shape tuning ---------------------------------------------------

// (twojmax, neighbour capacity in bands of 8, grid points in powers of two)
static uint64_t tune_key(int tj, int kmax, int64_t points) {
    int lg = 0;
    while (lg < 62 && (int64_t(1) << (lg + 1)) <= points) ++lg;
    return (uint64_t)tj | ((uint64_t)((kmax + 7) / 8) << 8) | ((uint64_t)lg << 24);
}

// one timed launch of each variant (CUDA events on the stream; the pass's
// first kernel launches are already queued before it)
template <class F>
static int time_variants(int n, float* ms, cudaStream_t st, F&& launch) {
    cudaEvent_t e[5];
    for (int i = 0; i <= n; ++i) MALA_CUDA_TRY(cudaEventCreate(&e[i]));
    cudaEventRecord(e[0], st);
    for (int v = 0; v < n; ++v) {
        launch(v);
        cudaEventRecord(e[v + 1], st);
    }
    cudaError_t err = cudaEventSynchronize(e[n]);
    for (int v = 0; v < n && err == cudaSuccess; ++v) err = cudaEventElapsedTime(&ms[v], e[v], e[v + 1]);
    for (int i = 0; i <= n; ++i) cudaEventDestroy(e[i]);
    if (err != cudaSuccess) return fail(MALA_ERR_CUDA, "variant timing failed: %s", cudaGetErrorString(err));
    return MALA_OK;
}

static int best_variant(const float* ms, int n) {
    int b = 0;
    for (int v = 1; v < n; ++v)
        if (ms[v] < ms[b]) b = v;
    return b;
}

// Tiles per chunk of the descriptor step (u half set, neighbour records and
// counts of a chunk stay below 4 GB) and the workspace sizes of a chunk.
struct DescSizes {
    int64_t chunk;
    size_t u, ab, cw, cnt;
};

static DescSizes desc_sizes(int64_t tiles, int tj, size_t e, int kmax) {
    DescSizes d;
    const int nh = n_half(tj);
    const size_t per_tile = (size_t)nh * 32 * 2 * e + (size_t)kmax * 32 * (5 * e) + 32 * sizeof(int);
    const size_t chunk_budget = (size_t)4 << 30;
    int64_t chunk = (int64_t)(chunk_budget / per_tile);
    if (chunk < 1) chunk = 1;
    if (chunk > tiles) chunk = tiles;
    d.chunk = chunk;
    // FP32 keeps tiles in pairs: room for an even number of tiles
    d.u = (size_t)((chunk + 1) & ~int64_t(1)) * nh * 32 * 2 * e;
    d.ab = (size_t)chunk * kmax * 32 * 4 * e;
    d.cw = (size_t)chunk * kmax * 32 * e;
    d.cnt = (size_t)chunk * 32 * sizeof(int);
    return d;
}

static int64_t snapshot_tiles(const mala_snapshot* s) {
    const int64_t tx = (s->grid[0] + kTileX - 1) / kTileX, ty = (s->grid[1] + kTileY - 1) / kTileY,
                  tz = (s->grid[2] + kTileZ - 1) / kTileZ;
    return tx * ty * tz;
}

void descriptors_ws_needs(Ctx* c, int n, const mala_snapshot* const* snaps, const mala_bispectrum_params* bp,
                          mala_precision prec, WsNeeds& out) {
    const size_t e = prec == MALA_MIXED ? 4 : 8;
    size_t staging = 0;
    int64_t tiles = 0;
    for (int i = 0; i < n; ++i) {
        staging += snapshot_ws_bytes(snaps[i], bp, bp->rcut);
        tiles += snapshot_tiles(snaps[i]);
    }
    out.add(c->ws_atoms, staging + 256);
    out.add(c->ws_batch, sizeof(BatchSnap) * n + 256);
    const DescSizes d = desc_sizes(tiles, bp->twojmax, e, c->kmax_hint);
    out.add(c->ws_u, d.u);
    out.add(c->ws_nbr_ab, d.ab);
    out.add(c->ws_nbr_c, d.cw);
    out.add(c->ws_nbr_cnt, d.cnt);
}

// Run neighbour search + compute_ui + compute_zi/bi over n snapshots in
// chunks of tiles.  The snapshots' tiles are numbered one after another, so a
// chunk (and each launch) may hold tiles of several snapshots; B rows are the
// snapshots' points in order (device, [sum P][nB]).  B and/or u_full (device,
// [P][n_full][2], a lone snapshot only) may be NULL.  dbg: optional neighbour-list
// output (a lone snapshot only).
template <class T>
static int run_descriptors(Ctx* c, int nsnap, const mala_snapshot* snaps, const mala_bispectrum_params* bp, T* B,
                           T* u_full, NbrOut* dbg, cudaStream_t st) {
    if (nsnap < 1) return fail(MALA_ERR_INVALID_ARG, "no snapshots");
    if ((u_full || dbg) && nsnap != 1) return fail(MALA_ERR_INVALID_ARG, "u or neighbour-list output needs one snapshot");
    // staging: one workspace region per snapshot
    std::vector<size_t> off(nsnap + 1, 0);
    for (int i = 0; i < nsnap; ++i) off[i + 1] = off[i] + snapshot_ws_bytes(&snaps[i], bp, bp->rcut);
    MALA_TRY(c->ws_atoms.reserve(c, off[nsnap] + 256));
    std::vector<BatchSnap> hb(nsnap);
    int64_t tiles = 0, rows = 0;
    for (int i = 0; i < nsnap; ++i) {
        MALA_TRY(stage_snapshot_at(&snaps[i], bp, bp->rcut, &hb[i].sd, c->ws_atoms.as<char>() + off[i], c, st));
        hb[i].tile_off = tiles;
        hb[i].row_off = rows;
        tiles += hb[i].sd.g.n_tiles;
        rows += hb[i].sd.g.P;
    }
    MALA_TRY(c->ws_batch.reserve(c, sizeof(BatchSnap) * nsnap + 256));
    BatchSnap* bs = c->ws_batch.as<BatchSnap>();
    // pinned staging of the table: the copy is ordered on the stream like the kernels
    if (c->host_batch_len < (size_t)nsnap) {
        if (c->host_batch) cudaFreeHost(c->host_batch);
        c->host_batch = nullptr;
        c->host_batch_len = 0;
        MALA_CUDA_TRY(cudaMallocHost(&c->host_batch, sizeof(BatchSnap) * nsnap));
        c->host_batch_len = nsnap;
    }
    MALA_CUDA_TRY(cudaStreamSynchronize(st));  // the previous table copy has been consumed
    memcpy(c->host_batch, hb.data(), sizeof(BatchSnap) * nsnap);  // BatchSnap is trivially copyable
    MALA_CUDA_TRY(cudaMemcpyAsync(bs, c->host_batch, sizeof(BatchSnap) * nsnap, cudaMemcpyHostToDevice, st));
    const int tj = bp->twojmax;
    const int nh = n_half(tj);
    const bool gauss_mode = dbg && dbg->gauss;  // Gaussian descriptors: no neighbour records
    int kmax = gauss_mode ? 0 : c->kmax_hint;
    for (int attempt = 0; attempt < 3; ++attempt) {
        const DescSizes ds = desc_sizes(tiles, tj, sizeof(T), kmax);
        const int64_t chunk = ds.chunk;
        MALA_TRY(c->ws_u.reserve(c, ds.u));
        MALA_TRY(c->ws_nbr_ab.reserve(c, ds.ab));
        MALA_TRY(c->ws_nbr_c.reserve(c, ds.cw));
        MALA_TRY(c->ws_nbr_cnt.reserve(c, ds.cnt));
        NbrOut nb;
        nb.ab = c->ws_nbr_ab.ptr;
        nb.cw = c->ws_nbr_c.ptr;
        nb.cnt = c->ws_nbr_cnt.as<int>();
        nb.kmax = kmax;
        if (dbg) {
            nb.dbg_atoms = dbg->dbg_atoms;
            nb.dbg_shifts = dbg->dbg_shifts;
            nb.dbg_counts = dbg->dbg_counts;
            nb.dbg_cap = dbg->dbg_cap;
            nb.gauss = dbg->gauss;
            nb.gauss_inv2s2 = dbg->gauss_inv2s2;
        }
        for (int i = 0; i < nsnap; ++i) MALA_CUDA_TRY(cudaMemsetAsync(hb[i].sd.maxcnt, 0, sizeof(int), st));
        // the kernel shapes of this pass: tuned per key, the defaults, or forced
        int v_ui = 0, v_zb = 0;
        bool tune_now = false;
        uint64_t key = 0;
        Ctx* rt = c->root();
        if (sizeof(T) == 4 && !gauss_mode && B) {
            std::lock_guard<std::mutex> lk(rt->tune_mu);
            if (rt->tune_mode == 2) {
                v_ui = rt->force_ui;
                v_zb = rt->force_zb;
            } else if (rt->tune_mode == 1) {
                key = tune_key(tj, kmax, rows);
                auto it = rt->tune.find(key);
                if (it != rt->tune.end()) {
                    v_ui = it->second.ui;
                    v_zb = it->second.zb;
                } else if (!c->parent) {
                    // only a synchronous call tunes: a serving slot shares the GPU with the other slots,
                    // so its timings would rank the variants by what else happened to run; slots take
                    // the defaults until a synchronous call has tuned the key
                    tune_now = true;
                }
            }
        }
        for (int64_t t0 = 0; t0 < tiles; t0 += chunk) {
            const int64_t nt = (tiles - t0) < chunk ? (tiles - t0) : chunk;
            if (sizeof(T) == 4)
                MALA_PROF(c, "k_neighbors", st, launch_neighbors(bs, nsnap, bp->rcut, bp->rfac0, bp->rmin0, t0, nt, nb, st));
            else
                MALA_PROF(c, "k_neighbors", st,
                          launch_neighbors_f64(bs, nsnap, bp->rcut, bp->rfac0, bp->rmin0, t0, nt, nb, st));
            if (B || u_full) {
                T* uh = c->ws_u.as<T>();
                if (tune_now) {
                    // every variant on this chunk's own data (they give the same bits), the fastest kept
                    TuneEntry e;
                    MALA_TRY(time_variants(ui_variant_count(true), e.ui_ms, st, [&](int v) {
                        launch_ui<T>(tj, nb, bp->wself, nt, uh, st, v);
                    }));
                    e.ui = best_variant(e.ui_ms, ui_variant_count(true));
                    launch_ui<T>(tj, nb, bp->wself, nt, uh, st, e.ui);
                    MALA_TRY(time_variants(zb_variant_count(), e.zb_ms, st, [&](int v) {
                        launch_zb<T>(c, tj, uh, bs, nsnap, t0, nt, nb.cnt, bp->wself, B, st, v);
                    }));
                    e.zb = best_variant(e.zb_ms, zb_variant_count());
                    v_ui = e.ui;
                    v_zb = e.zb;
                    tune_now = false;
                    std::lock_guard<std::mutex> lk(rt->tune_mu);
                    rt->tune[key] = e;
                } else {
                    MALA_PROF(c, "k_ui", st, launch_ui<T>(tj, nb, bp->wself, nt, uh, st, v_ui));
                    if (B)
                        MALA_PROF(c, "k_zb", st,
                                  launch_zb<T>(c, tj, uh, bs, nsnap, t0, nt, nb.cnt, bp->wself, B, st, v_zb));
                }
                if (u_full) MALA_PROF(c, "k_u_expand", st, launch_u_expand<T>(tj, uh, hb[0].sd.g, t0, nt, u_full, st));
            }
        }
        MALA_CUDA_TRY(cudaGetLastError());
        // per snapshot: max neighbour count, species flag
        std::vector<int> flags(2 * (size_t)nsnap);
        for (int i = 0; i < nsnap; ++i)
            MALA_CUDA_TRY(cudaMemcpyAsync(&flags[2 * i], hb[i].sd.maxcnt, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
        MALA_CUDA_TRY(cudaMemcpyAsync(c->host_ints + 2, c->tables.err_d, sizeof(int), cudaMemcpyDeviceToHost, st));
        MALA_CUDA_TRY(cudaStreamSynchronize(st));
        int maxcnt = 0;
        for (int i = 0; i < nsnap; ++i) {
            if (flags[2 * i + 1]) return fail(MALA_ERR_INVALID_ARG, "species index outside 0..n_species-1 (snapshot %d)", i);
            maxcnt = std::max(maxcnt, flags[2 * i]);
        }
        if (c->host_ints[2]) {
            const int code = c->host_ints[2];
            cudaMemsetAsync(c->tables.err_d, 0, sizeof(int), st);
            if (code == 2) return fail(MALA_ERR_TIMEOUT, "compute_zi/bi: a copy into shared memory did not complete in time");
            return fail(MALA_ERR_UNSUPPORTED, "a bispectrum partial sum exceeded 1e8 (outside the fixed-point range)");
        }
        if (dbg) dbg->kmax = maxcnt;
        if (gauss_mode) return MALA_OK;
        if (maxcnt <= kmax) {
            if (maxcnt > c->kmax_hint) c->kmax_hint = maxcnt;
            return MALA_OK;
        }
        kmax = (maxcnt + 7) & ~7;
        c->kmax_hint = kmax;
    }
    return fail(MALA_ERR_UNSUPPORTED, "neighbour capacity could not be established");
}

int snap_descriptors_full(Ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, void* B,
                          void* u_full, NbrOut* nl, mala_precision prec, cudaStream_t st) {
    if (prec == MALA_MIXED) return run_descriptors<float>(c, 1, snap, bp, (float*)B, (float*)u_full, nl, st);
    return run_descriptors<double>(c, 1, snap, bp, (double*)B, (double*)u_full, nl, st);
}

int snap_descriptors(Ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, void* B, void* u_full,
                     mala_precision prec, cudaStream_t st) {
    if (prec == MALA_MIXED) return run_descriptors<float>(c, 1, snap, bp, (float*)B, (float*)u_full, nullptr, st);
    return run_descriptors<double>(c, 1, snap, bp, (double*)B, (double*)u_full, nullptr, st);
}

int snap_gaussian(Ctx* c, const mala_snapshot* snap, double rcut, double sigma, void* G, mala_precision prec,
                  cudaStream_t st) {
    mala_bispectrum_params bp = {0, rcut, 0.99363, 0.0, 1.0, 0, nullptr};
    NbrOut gd;
    gd.gauss = G;
    gd.gauss_inv2s2 = 1.0 / (2.0 * sigma * sigma);
    if (prec == MALA_MIXED) return run_descriptors<float>(c, 1, snap, &bp, nullptr, nullptr, &gd, st);
    return run_descriptors<double>(c, 1, snap, &bp, nullptr, nullptr, &gd, st);
}

int snap_descriptors_batch(Ctx* c, int n, const mala_snapshot* snaps, const mala_bispectrum_params* bp, void* B,
                           mala_precision prec, cudaStream_t st) {
    if (prec == MALA_MIXED) return run_descriptors<float>(c, n, snaps, bp, (float*)B, nullptr, nullptr, st);
    return run_descriptors<double>(c, n, snaps, bp, (double*)B, nullptr, nullptr, st);
}

// ---- per-kernel event timing ---------------------------------------------

int prof_begin(Ctx* c, const char* name, cudaStream_t st) {
    if (!c->prof.on) return -1;
    std::lock_guard<std::mutex> lk(c->prof_mu);
    Prof::Rec r;
    r.name = name;
    for (cudaEvent_t* e : {&r.a, &r.b}) {
        if (!c->prof.pool.empty()) {
            *e = c->prof.pool.back();
            c->prof.pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            return -1;
        }
    }
    cudaEventRecord(r.a, st);
    c->prof.pending.push_back(r);
    return (int)c->prof.pending.size() - 1;
}

void prof_end(Ctx* c, int idx, cudaStream_t st) {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(c->prof_mu);
    if (idx < (int)c->prof.pending.size()) cudaEventRecord(c->prof.pending[idx].b, st);
}

static void prof_collect(Ctx* c) {
    std::lock_guard<std::mutex> lk(c->prof_mu);
    for (auto& r : c->prof.pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto& t = c->prof.total[r.name];
            t.first += ms;
            t.second += 1;
        }
        c->prof.pool.push_back(r.a);
        c->prof.pool.push_back(r.b);
    }
    c->prof.pending.clear();
}

}  // namespace mala

using namespace mala;

struct mala_ctx : public mala::Ctx {};
struct mala_model : public mala::Model {};

extern "C" {

int mala_version(void) { return 1; }

const char* mala_last_error(void) { return mala::g_err; }

int mala_create(mala_ctx** out, int device, size_t hbm_budget_bytes) {
    if (!out) return fail(MALA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(MALA_ERR_CUDA, "no CUDA device available: %s", cudaGetErrorString(e));
    }
    if (device < 0 || device >= ndev) return fail(MALA_ERR_INVALID_ARG, "device %d out of range", device);
    MALA_DEVICE_SCOPE(device);
    cudaDeviceProp prop;
    MALA_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10) return fail(MALA_ERR_UNSUPPORTED, "device %s (sm_%d%d) is not a Blackwell GPU", prop.name, prop.major, prop.minor);
    auto* c = new mala_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    c->num_sms = prop.multiProcessorCount;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&c->host_ints, 64 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->host_scalars, 64 * sizeof(double)) != cudaSuccess) {
        delete c;
        return fail(MALA_ERR_CUDA, "stream / pinned buffer creation failed");
    }
    int rc = upload_cg_tables(c);
    if (rc == MALA_OK) rc = upload_polylog_tables();
    if (rc == MALA_OK) rc = upload_ui_tables();
    if (rc != MALA_OK) {
        mala_destroy(c);
        return rc;
    }
    *out = c;
    return MALA_OK;
}

void mala_destroy(mala_ctx* c) {
    if (!c) return;
    DeviceScope dev_scope(c->device);
    server_stop(c);
    cudaDeviceSynchronize();
    {
        // networks outliving their context keep only their host object
        std::lock_guard<std::mutex> lk(c->models_mu);
        for (Model* m : c->models) {
            model_free(m);
            m->ctx = nullptr;
        }
        c->models.clear();
    }
    prof_collect(c);
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->host_ints) cudaFreeHost(c->host_ints);
    if (c->host_scalars) cudaFreeHost(c->host_scalars);
    if (c->host_dos) cudaFreeHost(c->host_dos);
    if (c->host_batch) cudaFreeHost(c->host_batch);
    delete c;
}

size_t mala_device_bytes(const mala_ctx* c) { return c ? (size_t)c->used : 0; }

int mala_profile(mala_ctx* c, int enable) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    prof_collect(c);
    if (enable) c->prof.total.clear();
    c->prof.on = enable != 0;
    return MALA_OK;
}

int mala_profile_get(mala_ctx* c, const char* kernel, double* total_ms, int64_t* launches) {
    if (!c || !kernel) return fail(MALA_ERR_INVALID_ARG, "bad arguments");
    prof_collect(c);
    if (strcmp(kernel, "all") == 0) {
        double ms = 0.0;
        int64_t n = 0;
        for (auto& kv : c->prof.total) {
            ms += kv.second.first;
            n += kv.second.second;
        }
        if (total_ms) *total_ms = ms;
        if (launches) *launches = n;
        return MALA_OK;
    }
    auto it = c->prof.total.find(kernel);
    if (total_ms) *total_ms = it == c->prof.total.end() ? 0.0 : it->second.first;
    if (launches) *launches = it == c->prof.total.end() ? 0 : it->second.second;
    return MALA_OK;
}

int mala_set_tuning(mala_ctx* c, int mode, int ui_variant, int zb_variant) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    if (mode < 0 || mode > 2) return fail(MALA_ERR_INVALID_ARG, "tuning mode %d is not 0, 1 or 2", mode);
    if (mode == 2 && (ui_variant < 0 || ui_variant >= ui_variant_count(true) || zb_variant < 0 ||
                      zb_variant >= zb_variant_count()))
        return fail(MALA_ERR_INVALID_ARG, "variant (%d, %d) outside [0, %d) x [0, %d)", ui_variant, zb_variant,
                    ui_variant_count(true), zb_variant_count());
    std::lock_guard<std::mutex> lk(c->tune_mu);
    c->tune_mode = mode;
    c->force_ui = mode == 2 ? ui_variant : 0;
    c->force_zb = mode == 2 ? zb_variant : 0;
    if (mode != 1) c->tune.clear();
    return MALA_OK;
}

int mala_tuning_variants(int32_t* n_ui, int32_t* n_zb) {
    if (n_ui) *n_ui = ui_variant_count(true);
    if (n_zb) *n_zb = zb_variant_count();
    return MALA_OK;
}

int mala_tuning_report(mala_ctx* c, char* buf, size_t len) {
    if (!c || !buf || len == 0) return fail(MALA_ERR_INVALID_ARG, "bad arguments");
    std::string out;
    std::lock_guard<std::mutex> lk(c->tune_mu);
    char line[512];
    for (auto& kv : c->tune) {
        const uint64_t k = kv.first;
        const TuneEntry& e = kv.second;
        int seg = 0, warps = 0;
        ui_variant_shape(e.ui, &seg, &warps);
        int n = snprintf(line, sizeof(line), "twojmax=%d kmax<=%d points~2^%d: compute_ui seg %d x %d warps (",
                         (int)(k & 0xff), (int)(((k >> 8) & 0xffff) * 8), (int)(k >> 24), seg, warps);
        for (int v = 0; v < ui_variant_count(true); ++v) {
            ui_variant_shape(v, &seg, &warps);
            n += snprintf(line + n, sizeof(line) - n, "%s%dx%d %.3f ms", v ? ", " : "", seg, warps, e.ui_ms[v]);
        }
        n += snprintf(line + n, sizeof(line) - n, "), compute_zi/bi %d warps (", zb_variant_warps(e.zb));
        for (int v = 0; v < zb_variant_count(); ++v)
            n += snprintf(line + n, sizeof(line) - n, "%s%d %.3f ms", v ? ", " : "", zb_variant_warps(v), e.zb_ms[v]);
        snprintf(line + n, sizeof(line) - n, ")\n");
        out += line;
    }
    snprintf(buf, len, "%s", out.c_str());
    return MALA_OK;
}

int mala_neighbor_lists(mala_ctx* c, const mala_snapshot* snap, double rcut, int32_t cap, int32_t* counts_dev,
                        int32_t* atoms_dev, int32_t* shifts_dev, int32_t* max_count, void* stream) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    MALA_TRY(check_snapshot(snap));
    if (!(rcut > 0.0)) return fail(MALA_ERR_INVALID_ARG, "rcut must be > 0");
    if (cap < 0 || (cap > 0 && (!atoms_dev || !shifts_dev)) || !counts_dev)
        return fail(MALA_ERR_INVALID_ARG, "bad neighbour-list output arguments");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    mala_bispectrum_params bp = {0, rcut, 0.99363, 0.0, 1.0, 0, nullptr};
    NbrOut dbg;
    dbg.dbg_atoms = atoms_dev;
    dbg.dbg_shifts = shifts_dev;
    dbg.dbg_counts = counts_dev;
    dbg.dbg_cap = cap;
    int rc = run_descriptors<float>(c, 1, snap, &bp, nullptr, nullptr, &dbg, as_stream(stream));
    if (rc == MALA_OK && max_count) *max_count = dbg.kmax;
    return rc;
}

int mala_descriptors(mala_ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, void* B_dev,
                     mala_precision precision, void* stream) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    MALA_TRY(check_snapshot(snap));
    MALA_TRY(check_bparams(bp));
    if (!B_dev) return fail(MALA_ERR_INVALID_ARG, "B output is NULL");
    if (precision != MALA_MIXED && precision != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return snap_descriptors(c, snap, bp, B_dev, nullptr, precision, as_stream(stream));
}

int mala_descriptors_batch(mala_ctx* c, int32_t n, const mala_snapshot* snaps, const mala_bispectrum_params* bp,
                           void* B_dev, mala_precision precision, void* stream) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    if (n < 1 || !snaps) return fail(MALA_ERR_INVALID_ARG, "need n >= 1 snapshots");
    for (int i = 0; i < n; ++i) MALA_TRY(check_snapshot(&snaps[i]));
    MALA_TRY(check_bparams(bp));
    if (!B_dev) return fail(MALA_ERR_INVALID_ARG, "B output is NULL");
    if (precision != MALA_MIXED && precision != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return snap_descriptors_batch(c, n, snaps, bp, B_dev, precision, as_stream(stream));
}

int mala_gaussian_descriptors(mala_ctx* c, const mala_snapshot* snap, double rcut, double sigma, void* G_dev,
                              mala_precision precision, void* stream) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    MALA_TRY(check_snapshot(snap));
    if (!(rcut > 0.0) || !std::isfinite(rcut)) return fail(MALA_ERR_INVALID_ARG, "rcut must be > 0");
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(MALA_ERR_INVALID_ARG, "sigma must be > 0");
    if (!G_dev) return fail(MALA_ERR_INVALID_ARG, "output is NULL");
    if (precision != MALA_MIXED && precision != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return snap_gaussian(c, snap, rcut, sigma, G_dev, precision, as_stream(stream));
}

int mala_expansion_coefficients(mala_ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                                void* u_dev, mala_precision precision, void* stream) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    MALA_TRY(check_snapshot(snap));
    MALA_TRY(check_bparams(bp));
    if (!u_dev) return fail(MALA_ERR_INVALID_ARG, "u output is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return snap_descriptors(c, snap, bp, nullptr, u_dev, precision, as_stream(stream));
}

}  // extern "C"
