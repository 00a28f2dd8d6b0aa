// mala_internal.h -- host-side internals shared by the library's translation
// units: the context, workspace buffers, error reporting and kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <deque>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mala.h"

namespace mala {

// ---- error reporting ------------------------------------------------------

void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);

#define MALA_CUDA_TRY(expr)                                                                 \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::mala::fail(MALA_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,              \
                                cudaGetErrorString(e_), __FILE__, __LINE__);                \
    } while (0)

#define MALA_TRY(expr)              \
    do {                            \
        int s_ = (expr);            \
        if (s_ != MALA_OK) return s_; \
    } while (0)

// ---- current device ---------------------------------------------------------

// Makes `dev` the calling thread's current device for the scope of an entry
// point and makes the caller's previous device current again on return, so a
// caller working on another device is not silently switched.
struct DeviceScope {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};
#define MALA_DEVICE_SCOPE(dev)                    \
    ::mala::DeviceScope mala_dev_scope_(dev);     \
    MALA_CUDA_TRY(mala_dev_scope_.err)

// ---- device buffers ---------------------------------------------------------

struct Ctx;

// Claims n bytes of the root context's HBM budget in one atomic step (several
// serving slots grow their workspaces concurrently); false if they do not fit.
bool budget_claim(Ctx* root, size_t n);

// A growable device buffer accounted against the context's HBM budget.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    Ctx* owner = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf();
    int reserve(Ctx* ctx, size_t n);  // ensures capacity >= n bytes (contents not kept)
    void release();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Device workspace a call will reserve, buffer by buffer: serving admission
// counts the growth beyond what a slot's buffers already hold.
struct WsNeeds {
    std::vector<std::pair<DevBuf*, size_t>> v;
    void add(DevBuf& b, size_t n) {
        for (auto& x : v)
            if (x.first == &b) {
                x.second = std::max(x.second, n);
                return;
            }
        v.emplace_back(&b, n);
    }
    size_t total() const {
        size_t t = 0;
        for (auto& x : v) t += x.second;
        return t;
    }
    size_t growth() const {
        size_t g = 0;
        for (auto& x : v) {
            const size_t have = x.first->ptr ? x.first->bytes : 0;
            if (x.second > have) g += x.second - have;
        }
        return g;
    }
};

// ---- descriptor tables (host-built, uploaded once) -------------------------

struct SnapTables {
    // global Clebsch-Gordan table (kTJMax numbering), float and double copies
    std::vector<double> cg;                 // host
    double* cg_d = nullptr;                 // device double copy
    // per twojmax: triple ids assigned to each zb warp
    int zb_warps = 8;
    std::map<int, std::vector<int16_t>> warp_lists;  // [warps][max_len] with -1 padding
    std::map<int, int> warp_list_len;
    // FP32 zb work units (triple, row, m1 row) per supported twojmax (index tj/2)
    int4* tri_d = nullptr;              // per triple: (global id, first unit, unit count, column)
    unsigned short* units_d = nullptr;  // ma | m1a << 4 | twice << 8
    int tri_off[8] = {0};
    int tri_n[8] = {0};
    int unit_off[8] = {0};
    int* err_d = nullptr;  // device error flags [8]
};

// Per-kernel CUDA-event timing on the launching stream (mala_profile).
struct Prof {
    bool on = false;
    struct Rec {
        const char* name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<double, int64_t>> total;  // name -> (ms, launches)
};
int prof_begin(struct Ctx* c, const char* name, cudaStream_t st);
void prof_end(struct Ctx* c, int idx, cudaStream_t st);
#define MALA_PROF(c, name, st, stmt)                        \
    do {                                                    \
        int pi_ = ::mala::prof_begin((c), (name), (st));    \
        stmt;                                               \
        ::mala::prof_end((c), pi_, (st));                   \
    } while (0)

// Network uploaded once: BF16 padded copies + tensor maps for the
// tensor-core path, FP64 copies for the plain path.
struct Model {
    Ctx* ctx = nullptr;
    int n_layers = 0;
    std::vector<int> dims;
    float leaky_slope = 0.01f;
    double slope_d = 0.01;
    int activate_output = 0;
    bool mixed_ok = false;           // shape fits the tensor-core kernel
    std::vector<int> nparts;         // weight chunks (N parts) per layer
    std::vector<int> prow, pn0;      // [layer][2]: rows and first row of each part
    std::vector<CUtensorMap> maps;   // [layer][2] BF16 weights [Npad][Kpad], 128-byte swizzle, box = part rows
    std::vector<void*> allocs;
    // MIXED: bf16 weights [Npad][Kpad] per layer, N padded to 16, K + 2 padded to 64;
    // columns K and K + 1 hold the bias as a BF16 (high, low) pair
    std::vector<void*> Wbf;
    std::vector<int> Kpad, Npad;
    float* in_shift = nullptr;   // device fp32 [dims[0]] (0 if absent)
    float* in_scale = nullptr;   // device fp32 [dims[0]] (1 if absent)
    // FP64_PLAIN
    std::vector<double*> Wd, bd;
    double* in_shift_d = nullptr;
    double* in_scale_d = nullptr;
    size_t bytes = 0;
};

// tables of the descriptor adjoint (Y contraction lists) for one twojmax, in Ctx::ws_ftab
struct ForceTables {
    int tj = -1;
    int ncoup = 0, list_len = 0, nh = 0;
    size_t off[10] = {0};
};

// launch plan of the FP32 Y step (units per row and warp) for one twojmax, in Ctx::ws_yplan
struct YiPlanState {
    int tj = -1;
    int row0[4] = {0, 0, 0, 0}, nrows[4] = {0, 0, 0, 0};
    size_t off[5] = {0, 0, 0, 0, 0};  // rows, off, units, be_t, be_f in ws_yplan
};

// Tile-shape tuning: per key (twojmax, neighbour-capacity band, grid-size band)
// the compute_ui and compute_zi/bi variants chosen, with the times that chose them.
struct TuneEntry {
    int ui = 0, zb = 0;
    float ui_ms[4] = {0, 0, 0, 0}, zb_ms[4] = {0, 0, 0, 0};
};

struct SnapStage;  // per-call staging of one snapshot (atoms, bins, neighbours)

// One queued or running request of the serving loop.
struct Request;

struct Ctx {
    Ctx* parent = nullptr;  // serving slots are child contexts of the user's context
    int device = 0;
    size_t budget = 0;  // 0 = unlimited
    std::atomic<size_t> used{0};
    Ctx* root() { return parent ? parent : this; }
    // bytes of the root budget that serving admission set aside for this
    // context's workspace growth and that DevBuf::reserve has not drawn yet
    size_t held = 0;
    cudaStream_t stream = nullptr;  // internal work stream for synchronous helpers
    SnapTables tables;
    int num_sms = 0;
    // workspaces of the synchronous path
    DevBuf ws_atoms, ws_batch, ws_bins, ws_nbr_ab, ws_nbr_c, ws_nbr_cnt, ws_u, ws_misc, ws_B, ws_ldos,
        ws_dens, ws_dos, ws_tile_dos, ws_units, ws_mlp64, ws_red, ws_w, ws_mlp_in;
    // workspaces of the force path
    ForceTables ftab;
    YiPlanState yplan;
    DevBuf ws_yplan;
    DevBuf ws_ftab, ws_force_y, ws_force_aux, ws_force_u, ws_force_nbr, ws_force_beta, ws_force_mlp, ws_force_g,
        ws_force_bt, ws_ace;
    double* host_dos = nullptr;     // pinned [max N_E]
    size_t host_dos_len = 0;
    double* host_scalars = nullptr; // pinned small buffer
    int* host_ints = nullptr;       // pinned small buffer
    std::vector<double> batch_dos;  // host D(e) of every snapshot of the last mala_predict_batch
    void* host_batch = nullptr;     // pinned staging of the descriptor batch table
    size_t host_batch_len = 0;      // entries it holds
    std::mutex mu;                  // serialises synchronous calls on this context
    std::mutex prof_mu;
    Prof prof;
    int kmax_hint = 64;             // neighbour capacity that sufficed last time
    // tile-shape tuning (the root context's state serves its serving slots too)
    int tune_mode = 1;              // 0 defaults, 1 autotune, 2 forced variants
    int force_ui = 0, force_zb = 0;
    std::mutex tune_mu;
    std::map<uint64_t, TuneEntry> tune;
    // serving
    struct Server* server = nullptr;
    // networks created on this context; mala_destroy frees their device memory
    std::mutex models_mu;
    std::set<Model*> models;
};

// ---- kernel launchers (descriptor path) ------------------------------------

struct SnapGeom {
    int n_atoms;
    double L[3];
    int periodic[3];
    int grid[3];
    int64_t P;
    int tiles[3];
    int64_t n_tiles;
    int nb[3];        // bins per axis
    double bs[3];     // bin size per axis
    int n_bins;
};

struct SnapDev {
    SnapGeom g;
    double* wpos = nullptr;   // [3][n] wrapped positions (SoA)
    double* wsp = nullptr;    // [n] element weight (FP64; the FP32 path rounds it once)
    int* bin_of = nullptr;    // [n]
    int* bin_start = nullptr; // [n_bins + 1]
    int* bin_atoms = nullptr; // [n]
    int* bin_fill = nullptr;  // [n_bins]
    int* maxcnt = nullptr;    // [4] device counters (max count, overflow flags)
    double* gcoord = nullptr; // grid coordinates (i / N_d) L_d: [grid0] | [grid1] | [grid2]
    float* wposf = nullptr;   // [6][n] wrapped positions as float pairs: x_hi, y_hi, z_hi, x_lo, y_lo, z_lo
};

// One snapshot of a batch: its staged atoms and where its tiles and grid
// points sit in the batch's numbering (a lone snapshot is a batch of one).
struct BatchSnap {
    SnapDev sd;
    int64_t tile_off;  // first tile in the batch's tile numbering
    int64_t row_off;   // first row of its points in the batch's B / LDOS rows
};

// bytes of device workspace one snapshot's staging needs (rcut = the cutoff)
size_t snapshot_ws_bytes(const mala_snapshot* snap, const mala_bispectrum_params* bp, double rcut);
// stage one snapshot into the workspace at `base` (snapshot_ws_bytes long)
int stage_snapshot_at(const mala_snapshot* snap, const mala_bispectrum_params* bp, double rcut, SnapDev* sd,
                      char* base, Ctx* c, cudaStream_t st);

// neighbour records of every tile: ab[tile][k][32] float4 (Cayley-Klein a, b),
// cw[tile][k][32] float (w * f_c), cnt[tile][32]; optional debug output of the
// atom index / image shift in point-major order.
struct NbrOut {
    void* ab = nullptr;   // float4 (MIXED) or double4 (FP64_PLAIN) records
    void* cw = nullptr;   // float or double
    int* cnt = nullptr;
    int kmax = 0;
    // debug
    int* dbg_atoms = nullptr;  // [P][dbg_cap]
    int* dbg_shifts = nullptr; // [P][dbg_cap][3]
    int* dbg_counts = nullptr; // [P]
    int dbg_cap = 0;
    // Gaussian descriptors: when set, each point's sum of exp(-d^2 / (2 sigma^2))
    // over its neighbours goes to gauss[row] (float or double) instead of records
    void* gauss = nullptr;
    double gauss_inv2s2 = 0.0;  // 1 / (2 sigma^2)
};

// tiles [tile0, tile0 + ntiles) of the batch bs[0..nsnap) (device array)
void launch_neighbors(const BatchSnap* bs, int nsnap, double rcut, double rfac0, double rmin0, int64_t tile0,
                      int64_t ntiles, const NbrOut& out, cudaStream_t st);
void launch_neighbors_f64(const BatchSnap* bs, int nsnap, double rcut, double rfac0, double rmin0, int64_t tile0,
                          int64_t ntiles, const NbrOut& out, cudaStream_t st);

// u half storage [tile][n_half][32] complex; variant: a compiled (segment length,
// warps per CTA) shape of the FP32 kernel (0 = default), ignored for FP64
template <class T>
void launch_ui(int twojmax, const NbrOut& nb, double wself, int64_t ntiles, T* u_half, cudaStream_t st,
               int variant = 0);
int ui_variant_count(bool fp32);
void ui_variant_shape(int v, int* seg, int* warps);

// nbr_cnt: the chunk's neighbour counts [tile][32]; wself: the self-term weight;
// variant: the FP32 kernel's warps-per-CTA shape (0 = default), ignored for FP64
template <class T>
void launch_zb(Ctx* c, int twojmax, const T* u_half, const BatchSnap* bs, int nsnap, int64_t tile0, int64_t ntiles,
               const int* nbr_cnt, double wself, T* B, cudaStream_t st, int variant = 0);
template <>
void launch_zb<float>(Ctx* c, int twojmax, const float* u_half, const BatchSnap* bs, int nsnap, int64_t tile0,
                      int64_t ntiles, const int* nbr_cnt, double wself, float* B, cudaStream_t st, int variant);
template <>
void launch_zb<double>(Ctx* c, int twojmax, const double* u_half, const BatchSnap* bs, int nsnap, int64_t tile0,
                       int64_t ntiles, const int* nbr_cnt, double wself, double* B, cudaStream_t st, int variant);
int zb_variant_count();
int zb_variant_warps(int v);
// the alternate-warp-count FP32 kernel (its own translation unit) and its constant tables
constexpr int kZbWarpsAlt = 8;
void launch_zb_alt(Ctx* c, int twojmax, const float* u_half, const BatchSnap* bs, int nsnap, int64_t tile0,
                   int64_t ntiles, const int* nbr_cnt, double wself, float* B, cudaStream_t st);
int upload_zb_alt_cg(const float2* cg2, int bytes);
int upload_zb_alt_jp1(const float* jp1, int bytes, int offset);

template <class T>
void launch_u_expand(int twojmax, const T* u_half, const SnapGeom& g, int64_t tile0, int64_t ntiles,
                     T* u_full, cudaStream_t st);

int upload_cg_tables(Ctx* c);
int upload_polylog_tables();
int upload_ui_tables();
int upload_zb_lists_f64(const int* lists, int bytes);
int snap_descriptors(Ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, void* B,
                     void* u_full, mala_precision prec, cudaStream_t st);
// Gaussian descriptors G(r) of one snapshot into G (float for MIXED, double for FP64_PLAIN)
int snap_gaussian(Ctx* c, const mala_snapshot* snap, double rcut, double sigma, void* G, mala_precision prec,
                  cudaStream_t st);
// descriptors of n snapshots in one pass of launches; B rows concatenated in snapshot order
int snap_descriptors_batch(Ctx* c, int n, const mala_snapshot* snaps, const mala_bispectrum_params* bp, void* B,
                           mala_precision prec, cudaStream_t st);

// the batch's snapshot holding global tile t (bs sorted by tile_off, bs[0].tile_off = 0)
__device__ __forceinline__ int batch_find(const BatchSnap* bs, int n, int64_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bs[mid].tile_off <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---- network and integrals ---------------------------------------------------

int model_upload(Ctx* c, const mala_mlp_desc* d, Model* m);

// workspace of the descriptor step for n snapshots (neighbour capacity: the context's hint),
// of the network over P rows (dos: with the fused DOS partials) and of the integrals of P rows
void descriptors_ws_needs(Ctx* c, int n, const mala_snapshot* const* snaps, const mala_bispectrum_params* bp,
                          mala_precision prec, WsNeeds& out);
void mlp_ws_needs(Ctx* c, const Model* m, int64_t P, bool dos, mala_precision prec, WsNeeds& out);
void integrate_ws_needs(Ctx* c, int64_t P, int nE, mala_precision prec, WsNeeds& out);

// ---- force path --------------------------------------------------------------

double clebsch_gordan(int j1, int m1, int j2, int m2, int j, int m);  // twice-units
// descriptors with the full u and neighbour lists of one snapshot (nl.dbg_* outputs set by the caller)
int snap_descriptors_full(Ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, void* B,
                          void* u_full, NbrOut* nl, mala_precision prec, cudaStream_t st);
// FP32 Y step of the descriptor adjoint: y[p] = conj(Y) N over the full set (snap_yi.cu)
int yi_units(Ctx* c, int tj, const float* u_full, const float* beta, int nB, int64_t P, float* y, cudaStream_t st);
// F_host[n_atoms][3] = -sum_r sum_j beta[r][j] dB(r, j)/dR from the staged snapshot sd
template <class T>
int descriptor_adjoint(Ctx* c, const SnapDev& sd, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                       const T* u_full, const T* beta, const NbrOut& nl, double* F_host, cudaStream_t st);
// beta[P][n_B] = sum_e v[e] dLDOS[p][e]/dB[p][:] (v device [n_E]); float for MIXED, double for FP64_PLAIN
int mlp_backward(Ctx* c, const Model* m, const void* B, int64_t P, const double* v_dev, void* beta,
                 mala_precision prec, cudaStream_t st);
// ACE descriptors (ace.cu): parameter check, column count, descriptors from a staged snapshot and its
// complete neighbour lists (nl.dbg_*), out: [P][n_desc] float (MIXED) or double
int check_ace_params(const mala_ace_params* ap);
int ace_count(const mala_ace_params* ap);
int ace_from_lists(Ctx* c, const SnapDev& sd, const mala_snapshot* snap, const mala_ace_params* ap,
                   const NbrOut& nl, void* out, mala_precision prec, cudaStream_t st);
// dE_b/dD at fixed N_e for D = dV * dos_sum: g_dev[n_E] = gscale * dE_b/dD; *fermi, *mu_tilde (host)
int energy_gradient(Ctx* c, const double* dos_sum, double dV, const mala_energy_grid* eg, double gscale,
                    double* g_dev, double* fermi, double* mu_tilde, cudaStream_t st);
void server_stop(Ctx* c);
int integrate_noalloc(Ctx* c, const void* ldos, int64_t P, double volume, const mala_energy_grid* eg,
                      const double* dos_sum, void* density, double* dos_host, double* fermi, double* eb, double* ne,
                      double* ts, mala_precision prec, cudaStream_t st);
int electron_count_at(Ctx* c, const double* D_host, const mala_energy_grid* eg, double mu, double* out,
                      cudaStream_t st);
void model_free(Model* m);
int mlp_forward(Ctx* c, const Model* m, const void* B, int64_t P, void* ldos, double* dos_sum,
                mala_precision prec, cudaStream_t st);
// ts: the entropy term -tau S_s (eV) of Eqs. electronicentropyDOS / KSfreeenergy, may be NULL
int integrate(Ctx* c, const void* ldos, int64_t P, double volume, const mala_energy_grid* eg,
              const double* dos_sum, void* density, double* dos_host, double* fermi, double* eb,
              double* ne, double* ts, mala_precision prec, cudaStream_t st);

}  // namespace mala
