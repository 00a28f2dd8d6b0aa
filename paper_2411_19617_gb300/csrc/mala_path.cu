// mala_path.cu -- C ABI of the network and integral steps, the whole path
// (mala_predict) and the serving loop (mala_submit / mala_poll / mala_wait /
// mala_release).
//
// Serving.  A server owns a FIFO of requests (each a deep copy of its inputs)
// and a few worker slots.  A slot is a child context: its own CUDA stream,
// workspaces and pinned buffers, sharing the parent's tables and HBM budget
// accounting.  A worker takes the oldest queued request whose device memory
// (its outputs plus any workspace growth) fits in what the budget has left,
// allocates the request's outputs, runs descriptors -> network -> integrals on
// its stream and marks the request done; requests on different slots run
// concurrently on the GPU.  Outputs stay on the device until mala_release.
// Admission claims the outputs and the slot's workspace growth from the budget
// in one atomic step per request, and an old queue head is never bypassed.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>

#include "mala_internal.h"
#include "snap_common.cuh"

namespace mala {

int check_snapshot(const mala_snapshot* s);
int check_bparams(const mala_bispectrum_params* bp);

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

static int check_model_desc(const mala_mlp_desc* d) {
    if (!d) return fail(MALA_ERR_INVALID_ARG, "network descriptor is NULL");
    if (d->n_layers < 1 || d->n_layers > 16 || !d->dims || !d->W || !d->b)
        return fail(MALA_ERR_INVALID_ARG, "bad network descriptor");
    for (int l = 0; l <= d->n_layers; ++l)
        if (d->dims[l] < 1 || d->dims[l] > 65536) return fail(MALA_ERR_INVALID_ARG, "bad layer width %d", d->dims[l]);
    for (int l = 0; l < d->n_layers; ++l)
        if (!d->W[l] || !d->b[l]) return fail(MALA_ERR_INVALID_ARG, "layer %d weights are NULL", l);
    if (!std::isfinite(d->leaky_slope)) return fail(MALA_ERR_INVALID_ARG, "leaky slope is not finite");
    return MALA_OK;
}

static int check_egrid(const mala_energy_grid* eg) {
    if (!eg) return fail(MALA_ERR_INVALID_ARG, "energy grid is NULL");
    if (eg->n_E < 2 || eg->n_E > 4096) return fail(MALA_ERR_INVALID_ARG, "n_E = %d outside 2..4096", eg->n_E);
    if (!(eg->de_eV > 0.0) || !(eg->kT_eV > 0.0) || !std::isfinite(eg->e0_eV) || !std::isfinite(eg->n_electrons))
        return fail(MALA_ERR_INVALID_ARG, "energy grid needs de > 0, kT > 0 and finite e0, N_e");
    return MALA_OK;
}

static double cell_volume(const mala_snapshot* s) { return s->cell[0][0] * s->cell[1][1] * s->cell[2][2]; }

// descriptors -> LDOS -> integrals into the given device buffers
static int run_path(Ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, const Model* m,
                    const mala_energy_grid* eg, mala_precision prec, void* B, void* ldos, void* dens, double* dos_sum,
                    mala_result* res, double* dos_host, cudaStream_t st) {
    const int64_t P = (int64_t)snap->grid[0] * snap->grid[1] * snap->grid[2];
    MALA_TRY(snap_descriptors(c, snap, bp, B, nullptr, prec, st));
    MALA_TRY(mlp_forward(c, m, B, P, ldos, dos_sum, prec, st));
    double eF = 0.0, Eb = 0.0, Ne = 0.0;
    double TS = 0.0;
    int rc = integrate(c, ldos, P, cell_volume(snap), eg, dos_sum, dens, dos_host, &eF, &Eb, &Ne, &TS, prec, st);
    res->status = rc;
    res->n_B = n_triples(bp->twojmax);
    res->n_E = eg->n_E;
    res->n_points = P;
    res->fermi_eV = eF;
    res->band_energy_eV = Eb;
    res->electron_count = Ne;
    res->entropy_term_eV = TS;
    res->B_dev = B;
    res->ldos_dev = ldos;
    res->density_dev = dens;
    return rc;
}

static int check_path_args(const mala_snapshot* snap, const mala_bispectrum_params* bp, const Model* m,
                           const mala_energy_grid* eg, mala_precision prec) {
    MALA_TRY(check_snapshot(snap));
    MALA_TRY(check_bparams(bp));
    MALA_TRY(check_egrid(eg));
    if (!m) return fail(MALA_ERR_INVALID_ARG, "model is NULL");
    if (prec != MALA_MIXED && prec != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    if (m->dims[0] != n_triples(bp->twojmax))
        return fail(MALA_ERR_INVALID_ARG, "network input width %d != %d descriptors", m->dims[0], n_triples(bp->twojmax));
    if (m->dims[m->n_layers] != eg->n_E)
        return fail(MALA_ERR_INVALID_ARG, "network output width %d != n_E %d", m->dims[m->n_layers], eg->n_E);
    return MALA_OK;
}

static size_t path_output_bytes(int64_t P, int nB, int nE, mala_precision prec) {
    const size_t e = prec == MALA_MIXED ? 4 : 8, l = prec == MALA_MIXED ? 2 : 8;
    return (size_t)P * nB * e + (size_t)P * nE * l + (size_t)P * e + (size_t)nE * 8 + 4 * 256;
}

// descriptors -> LDOS -> integrals for n snapshots into the given device buffers
// (rows of snapshot i at row[i]): descriptors of all snapshots in one pass of
// launches, the network over all rows in one launch, the integrals per
// snapshot.  A lone snapshot takes its DOS column sums from the network's
// epilogue (dos_sum, may be NULL otherwise), so n = 1 is exactly run_path.
// dos_host[i]: host [n_E] per snapshot.  Returns the first per-snapshot
// failure other than MALA_ERR_FERMI_BRACKET, else the first bracket error,
// else MALA_OK; res[i].status holds each snapshot's own status.
static int run_path_batch(Ctx* c, int n, const mala_snapshot* const* snaps, const mala_bispectrum_params* bp,
                          const Model* m, const mala_energy_grid* const* egs, mala_precision prec, char* B, char* L,
                          char* D, double* dos_sum, double* const* dos_host, mala_result* const* res,
                          cudaStream_t st) {
    if (n == 1) return run_path(c, snaps[0], bp, m, egs[0], prec, B, L, D, dos_sum, res[0], dos_host[0], st);
    std::vector<int64_t> row(n + 1, 0);
    std::vector<mala_snapshot> sv(n);
    for (int i = 0; i < n; ++i) {
        sv[i] = *snaps[i];
        row[i + 1] = row[i] + (int64_t)snaps[i]->grid[0] * snaps[i]->grid[1] * snaps[i]->grid[2];
    }
    const int nB = n_triples(bp->twojmax), nE = egs[0]->n_E;
    const size_t e = prec == MALA_MIXED ? 4 : 8, l = prec == MALA_MIXED ? 2 : 8;
    MALA_TRY(snap_descriptors_batch(c, n, sv.data(), bp, B, prec, st));
    MALA_TRY(mlp_forward(c, m, B, row[n], L, nullptr, prec, st));
    int first_rc = MALA_OK;
    for (int i = 0; i < n; ++i) {
        const int64_t Pi = row[i + 1] - row[i];
        double eF = 0.0, Eb = 0.0, Ne = 0.0, TS = 0.0;
        const int rc = integrate(c, L + (size_t)row[i] * nE * l, Pi, cell_volume(snaps[i]), egs[i], nullptr,
                                 D + (size_t)row[i] * e, dos_host[i], &eF, &Eb, &Ne, &TS, prec, st);
        if (rc != MALA_OK && rc != MALA_ERR_FERMI_BRACKET) return rc;
        if (rc != MALA_OK && first_rc == MALA_OK) first_rc = rc;
        mala_result& r = *res[i];
        r.status = rc;
        r.n_B = nB;
        r.n_E = nE;
        r.n_points = Pi;
        r.fermi_eV = eF;
        r.band_energy_eV = Eb;
        r.electron_count = Ne;
        r.entropy_term_eV = TS;
        r.B_dev = B + (size_t)row[i] * nB * e;
        r.ldos_dev = L + (size_t)row[i] * nE * l;
        r.density_dev = D + (size_t)row[i] * e;
    }
    return first_rc;
}

// ---- serving ---------------------------------------------------------------

// device outputs of one served batch, shared by its requests until the last release
struct OutBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    int refs = 0;
};

struct Request {
    uint64_t ticket = 0;
    std::vector<double> pos;
    std::vector<int32_t> species;
    std::vector<double> weights;
    mala_snapshot snap{};
    mala_bispectrum_params bp{};
    mala_energy_grid eg{};
    const Model* model = nullptr;
    mala_precision prec = MALA_MIXED;
    int64_t P = 0;
    size_t out_bytes = 0;
    // results
    int state = 0;  // 0 queued, 1 running, 2 done
    int status = MALA_PENDING;
    std::string error;
    OutBuf* out = nullptr;  // the batch's outputs: B | LDOS | density rows of all its requests, then dos_sum
    std::vector<double> dos;
    mala_result res{};
    std::chrono::steady_clock::time_point t_submit, t_done;
};

struct Server {
    Ctx* root = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<std::unique_ptr<Ctx>> slots;
    std::vector<std::thread> workers;
    uint64_t next_ticket = 1;
    bool stop = false;
    int running = 0;
    std::vector<char> busy;          // per slot: a batch is running on it
    size_t out_live = 0;             // bytes of batch outputs allocated and not yet released
    cudaEvent_t t0 = nullptr;        // device-clock origin of the batches' intervals
};

// requests that may share one batch: same network, precision, bispectrum setting and n_E
static bool batchable(const Request* a, const Request* b) {
    if (a->model != b->model || a->prec != b->prec || a->eg.n_E != b->eg.n_E) return false;
    const mala_bispectrum_params &p = a->bp, &q = b->bp;
    if (p.twojmax != q.twojmax || p.rcut != q.rcut || p.rfac0 != q.rfac0 || p.rmin0 != q.rmin0 || p.wself != q.wself ||
        p.n_species != q.n_species || (p.weights == nullptr) != (q.weights == nullptr))
        return false;
    return a->weights == b->weights;
}

constexpr int kServeBatchMax = 16;                // requests per batch
constexpr int64_t kServeBatchPoints = 8000000;    // grid points per batch
constexpr double kServeBypassS = 0.05;            // how long later requests may pass a queue head that does not fit

// the path's workspaces of a serving slot
static std::array<DevBuf*, 17> slot_buffers(Ctx* s) {
    return {&s->ws_atoms, &s->ws_batch, &s->ws_bins, &s->ws_nbr_ab, &s->ws_nbr_c, &s->ws_nbr_cnt, &s->ws_u,
            &s->ws_misc, &s->ws_B, &s->ws_ldos, &s->ws_dens, &s->ws_dos, &s->ws_tile_dos, &s->ws_mlp64,
            &s->ws_red, &s->ws_w, &s->ws_mlp_in};
}

// an idle slot's workspaces, returned to the budget
static void release_workspaces(Ctx* s) {
    for (DevBuf* b : slot_buffers(s)) b->release();
}

static size_t workspace_bytes(Ctx* s) {
    size_t t = 0;
    for (DevBuf* b : slot_buffers(s)) t += b->ptr ? b->bytes : 0;
    return t;
}

// Device workspace a batch would add to a slot: the growth of the slot's
// buffers (descriptor chunk, network input, integrals) beyond what they hold
// (or, with total, all of it).
static size_t batch_ws_growth(Ctx* slot, const std::vector<Request*>& b, bool total = false) {
    const int n = (int)b.size();
    std::vector<const mala_snapshot*> snaps(n);
    int64_t P = 0;
    for (int i = 0; i < n; ++i) {
        snaps[i] = &b[i]->snap;
        P += b[i]->P;
    }
    WsNeeds w;
    descriptors_ws_needs(slot, n, snaps.data(), &b[0]->bp, b[0]->prec, w);
    mlp_ws_needs(slot, b[0]->model, P, n == 1, b[0]->prec, w);
    for (const Request* r : b) integrate_ws_needs(slot, r->P, r->eg.n_E, r->prec, w);
    return total ? w.total() : w.growth();
}

static void worker_loop(Server* sv, Ctx* slot, int idx) {
    cudaSetDevice(slot->device);
    for (;;) {
        std::vector<Request*> batch;
        size_t batch_bytes = 0, ws_grow = 0;
        bool over_budget = false;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stop) return;
                // The oldest queued request whose outputs and workspace growth fit in what the
                // budget has left, then every later compatible one while the batch still fits
                // (continuous batching).  The bytes are claimed from the budget one request at
                // a time; the workspace part is set aside for this slot's buffers.  A queue head
                // that does not fit may be passed by later requests only for kServeBypassS, after
                // which nothing is admitted until it fits (no starvation of large snapshots).
                Ctx* root = sv->root;
                int64_t pts = 0;
                const auto now = std::chrono::steady_clock::now();
                for (auto it = sv->queue.begin(); it != sv->queue.end();) {
                    Request* q = sv->reqs[*it].get();
                    const bool first = batch.empty();
                    if (!first && ((int)batch.size() >= kServeBatchMax || !batchable(batch[0], q) ||
                                   pts + q->P > kServeBatchPoints)) {
                        ++it;
                        continue;
                    }
                    batch.push_back(q);
                    const size_t out = batch_bytes + q->out_bytes;
                    const size_t grow = batch_ws_growth(slot, batch);
                    const size_t have = batch_bytes + ws_grow, need = out + grow;
                    bool fits = need <= have || budget_claim(root, need - have);
                    if (fits && need < have) root->used -= have - need;
                    if (!fits && first && (sv->running == 0 || it == sv->queue.begin())) {
                        // workspaces that idle slots keep from earlier batches may be what blocks the
                        // head: release them (the slots regrow them on their next batch) and try again
                        const double age = std::chrono::duration<double>(now - q->t_submit).count();
                        if (sv->running == 0 || age > kServeBypassS) {
                            for (size_t j = 0; j < sv->slots.size(); ++j)
                                if ((int)j != idx && !sv->busy[j]) release_workspaces(sv->slots[j].get());
                            const size_t grow2 = batch_ws_growth(slot, batch);
                            fits = budget_claim(root, q->out_bytes + grow2);
                            if (fits) {
                                batch_bytes = q->out_bytes;
                                ws_grow = grow2;
                                pts += q->P;
                                it = sv->queue.erase(it);
                                continue;
                            }
                        }
                    }
                    if (!fits) {
                        batch.pop_back();
                        if (first) {
                            if (sv->running == 0) {
                                // Nothing runs.  Outputs still held by finished requests come back when
                                // they are released and workspaces when slots are trimmed; what remains
                                // is memory the server cannot free.  A request that cannot fit even
                                // then is run alone to report the budget error; otherwise it waits.
                                size_t ws = 0;
                                for (auto& sl : sv->slots) ws += workspace_bytes(sl.get());
                                const size_t floor = root->used - std::min<size_t>(root->used, sv->out_live + ws);
                                std::vector<Request*> alone{q};
                                const size_t ever = q->out_bytes + batch_ws_growth(slot, alone, true);
                                if (root->budget && floor + ever > root->budget) {
                                    batch.push_back(q);
                                    it = sv->queue.erase(it);
                                    over_budget = true;
                                }
                                break;
                            }
                            const double age = std::chrono::duration<double>(now - q->t_submit).count();
                            if (it == sv->queue.begin() && age > kServeBypassS) break;  // the old head goes first
                            ++it;
                            continue;
                        }
                        break;
                    }
                    batch_bytes = out;
                    ws_grow = grow;
                    pts += q->P;
                    it = sv->queue.erase(it);
                }
                if (!batch.empty()) break;
                // woken by submissions, completions and releases; the timeout re-checks the head's age
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
            for (Request* r : batch) r->state = 1;
            ++sv->running;
            sv->busy[idx] = 1;
            slot->held = ws_grow;
            if (over_budget) batch_bytes = 0;  // nothing claimed or allocated: reported below
            sv->out_live += batch_bytes;
        }
        int rc = MALA_OK;
        const int n = (int)batch.size();
        OutBuf* ob = nullptr;
        if (batch_bytes == 0) {
            rc = fail(MALA_ERR_OOM, "request of %zu bytes does not fit in the HBM budget", batch[0]->out_bytes);
        } else {
            ob = new OutBuf();
            ob->bytes = batch_bytes;
            ob->refs = n;
            if (cudaMalloc(&ob->ptr, batch_bytes) != cudaSuccess) {
                cudaGetLastError();
                ob->ptr = nullptr;
                rc = fail(MALA_ERR_OOM, "cudaMalloc(%zu) for request outputs failed", batch_bytes);
            }
        }
        if (rc == MALA_OK) {
            // carve: B rows | LDOS rows | density rows of all requests, then each request's dos_sum
            const Request* r0 = batch[0];
            const size_t e = r0->prec == MALA_MIXED ? 4 : 8, l = r0->prec == MALA_MIXED ? 2 : 8;
            const int nB = n_triples(r0->bp.twojmax), nE = r0->eg.n_E;
            int64_t P = 0;
            for (Request* r : batch) P += r->P;
            auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
            char* p = static_cast<char*>(ob->ptr);
            char* B = p;
            p += al((size_t)P * nB * e);
            char* L = p;
            p += al((size_t)P * nE * l);
            char* D = p;
            p += al((size_t)P * e);
            double* S = reinterpret_cast<double*>(p);
            std::vector<const mala_snapshot*> snaps(n);
            std::vector<const mala_energy_grid*> egs(n);
            std::vector<double*> dh(n);
            std::vector<mala_result*> res(n);
            for (int i = 0; i < n; ++i) {
                Request* r = batch[i];
                r->dos.assign(nE, 0.0);
                snaps[i] = &r->snap;
                egs[i] = &r->eg;
                dh[i] = r->dos.data();
                res[i] = &r->res;
            }
            std::lock_guard<std::mutex> lk(slot->mu);
            cudaEvent_t ea = nullptr, eb = nullptr;
            const bool timed = sv->t0 && cudaEventCreate(&ea) == cudaSuccess && cudaEventCreate(&eb) == cudaSuccess;
            if (timed) cudaEventRecord(ea, slot->stream);
            rc = run_path_batch(slot, n, snaps.data(), &r0->bp, r0->model, egs.data(), r0->prec, B, L, D, S, dh.data(),
                                res.data(), slot->stream);
            if (timed) {
                cudaEventRecord(eb, slot->stream);
                float a = 0.f, b = 0.f;
                if (cudaEventSynchronize(eb) == cudaSuccess && cudaEventElapsedTime(&a, sv->t0, ea) == cudaSuccess &&
                    cudaEventElapsedTime(&b, sv->t0, eb) == cudaSuccess)
                    for (mala_result* rr : res) {
                        rr->gpu_start_ms = a;
                        rr->gpu_end_ms = b;
                    }
                cudaGetLastError();
            }
            if (ea) cudaEventDestroy(ea);
            if (eb) cudaEventDestroy(eb);
        }
        // workspace bytes set aside for this batch and not drawn by the slot's buffers go back
        sv->root->used -= slot->held;
        slot->held = 0;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            const std::string err = rc != MALA_OK ? std::string(mala_last_error()) : std::string();
            const auto now = std::chrono::steady_clock::now();
            for (Request* r : batch) {
                // per-request status: its own bracket result inside a good batch, else the batch's error
                const int st = (rc == MALA_OK || rc == MALA_ERR_FERMI_BRACKET) && ob ? r->res.status : rc;
                r->status = st;
                if (st != MALA_OK) r->error = st == rc ? err : std::string("N(mu) - N_e has no sign change");
                r->out = ob;
                r->t_done = now;
                r->res.status = st;
                r->res.dos = r->dos.empty() ? nullptr : r->dos.data();
                r->res.submit_to_done_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
                r->state = 2;
            }
            --sv->running;
            sv->busy[idx] = 0;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

static int server_start(Ctx* c) {
    if (c->server) return MALA_OK;
    auto* sv = new Server();
    sv->root = c;
    int nslots = 4;
    if (const char* e = getenv("MALA_SERVE_SLOTS")) nslots = std::max(1, std::min(16, atoi(e)));
    for (int i = 0; i < nslots; ++i) {
        auto s = std::make_unique<Ctx>();
        s->parent = c;
        s->device = c->device;
        s->num_sms = c->num_sms;
        s->tables = c->tables;
        s->kmax_hint = c->kmax_hint;
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&s->host_ints, 64 * sizeof(int)) != cudaSuccess ||
            cudaMallocHost(&s->host_scalars, 64 * sizeof(double)) != cudaSuccess) {
            delete sv;
            return fail(MALA_ERR_CUDA, "could not create a serving slot");
        }
        sv->slots.push_back(std::move(s));
    }
    sv->busy.assign(sv->slots.size(), 0);
    if (cudaEventCreate(&sv->t0) == cudaSuccess) cudaEventRecord(sv->t0, c->stream);
    else sv->t0 = nullptr;
    for (size_t i = 0; i < sv->slots.size(); ++i) sv->workers.emplace_back(worker_loop, sv, sv->slots[i].get(), (int)i);
    c->server = sv;
    return MALA_OK;
}

void server_stop(Ctx* c) {
    Server* sv = c->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    std::vector<OutBuf*> outs;
    for (auto& kv : sv->reqs)
        if (kv.second->out && std::find(outs.begin(), outs.end(), kv.second->out) == outs.end())
            outs.push_back(kv.second->out);
    for (OutBuf* ob : outs) {
        if (ob->ptr) cudaFree(ob->ptr);
        c->used -= ob->bytes;
        delete ob;
    }
    if (sv->t0) cudaEventDestroy(sv->t0);
    for (auto& s : sv->slots) {
        cudaStreamSynchronize(s->stream);
        cudaStreamDestroy(s->stream);
        cudaFreeHost(s->host_ints);
        cudaFreeHost(s->host_scalars);
        if (s->host_dos) cudaFreeHost(s->host_dos);
        if (s->host_batch) cudaFreeHost(s->host_batch);
    }
    delete sv;
    c->server = nullptr;
}

// ---- forces (Eqs. forces / forcesmala with E = E_b) --------------------------

// descriptors of one snapshot with the full u (ws_force_u) and complete
// neighbour lists (ws_force_nbr: counts[P] | atoms[P][cap] | shifts[P][cap][3]);
// the capacity grows until every list fits.  B may be NULL.
static int stage_force_descriptors(Ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                                   mala_precision prec, void* B, NbrOut* nl, cudaStream_t st) {
    const int64_t P = (int64_t)snap->grid[0] * snap->grid[1] * snap->grid[2];
    const size_t e = prec == MALA_MIXED ? 4 : 8;
    MALA_TRY(c->ws_force_u.reserve(c, e * 2 * (size_t)n_full(bp->twojmax) * (size_t)std::max<int64_t>(P, 1) + 256));
    int cap = std::max(32, (c->kmax_hint + 7) & ~7);
    for (int attempt = 0; attempt < 3; ++attempt) {
        const size_t Pp = (size_t)((P + 63) & ~int64_t(63));
        MALA_TRY(c->ws_force_nbr.reserve(c, sizeof(int) * Pp * (1 + 4 * (size_t)cap) + 256));
        NbrOut d;
        d.dbg_counts = c->ws_force_nbr.as<int>();
        d.dbg_atoms = d.dbg_counts + Pp;
        d.dbg_shifts = d.dbg_atoms + Pp * cap;
        d.dbg_cap = cap;
        MALA_TRY(snap_descriptors_full(c, snap, bp, B, c->ws_force_u.ptr, &d, prec, st));
        if (d.kmax <= cap) {
            *nl = d;
            return MALA_OK;
        }
        cap = (d.kmax + 7) & ~7;
    }
    return fail(MALA_ERR_UNSUPPORTED, "neighbour-list capacity for the force step could not be established");
}

// complete neighbour lists of one snapshot (no descriptors) into ws_force_nbr
static int stage_lists_only(Ctx* c, const mala_snapshot* snap, double rcut, int n_species, NbrOut* nl,
                            cudaStream_t st) {
    const int64_t P = (int64_t)snap->grid[0] * snap->grid[1] * snap->grid[2];
    mala_bispectrum_params bp = {0, rcut, 0.99363, 0.0, 1.0, n_species, nullptr};
    int cap = std::max(32, (c->kmax_hint + 7) & ~7);
    for (int attempt = 0; attempt < 3; ++attempt) {
        const size_t Pp = (size_t)((P + 63) & ~int64_t(63));
        MALA_TRY(c->ws_force_nbr.reserve(c, sizeof(int) * Pp * (1 + 4 * (size_t)cap) + 256));
        NbrOut d;
        d.dbg_counts = c->ws_force_nbr.as<int>();
        d.dbg_atoms = d.dbg_counts + Pp;
        d.dbg_shifts = d.dbg_atoms + Pp * cap;
        d.dbg_cap = cap;
        MALA_TRY(snap_descriptors_full(c, snap, &bp, nullptr, nullptr, &d, MALA_MIXED, st));
        if (d.kmax <= cap) {
            *nl = d;
            return MALA_OK;
        }
        cap = (d.kmax + 7) & ~7;
    }
    return fail(MALA_ERR_UNSUPPORTED, "neighbour-list capacity could not be established");
}

static int adjoint_of_staged(Ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, mala_precision prec,
                             const void* beta, const NbrOut& nl, double* F, cudaStream_t st) {
    const SnapDev& sd = static_cast<const BatchSnap*>(c->host_batch)[0].sd;
    if (prec == MALA_MIXED)
        return descriptor_adjoint<float>(c, sd, snap, bp, c->ws_force_u.as<float>(), static_cast<const float*>(beta),
                                         nl, F, st);
    return descriptor_adjoint<double>(c, sd, snap, bp, c->ws_force_u.as<double>(), static_cast<const double*>(beta),
                                      nl, F, st);
}

}  // namespace mala

using namespace mala;

struct mala_ctx : public mala::Ctx {};
struct mala_model : public mala::Model {};

extern "C" {

int mala_model_create(mala_ctx* c, const mala_mlp_desc* desc, mala_model** out) {
    if (!c || !out) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    MALA_TRY(check_model_desc(desc));
    MALA_DEVICE_SCOPE(c->device);
    auto* m = new mala_model();
    int rc = model_upload(c, desc, m);
    if (rc != MALA_OK) {
        model_free(m);
        delete m;
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(c->models_mu);
        c->models.insert(m);
    }
    *out = m;
    return MALA_OK;
}

void mala_model_destroy(mala_model* m) {
    if (!m) return;
    if (Ctx* c = m->ctx) {
        {
            std::lock_guard<std::mutex> lk(c->models_mu);
            c->models.erase(m);
        }
        model_free(m);
    }
    delete m;
}

int mala_ldos_forward(mala_ctx* c, const mala_model* m, const void* B_dev, int64_t P, void* ldos_dev,
                      double* dos_sum_dev, mala_precision precision, void* stream) {
    if (!c || !m || (!B_dev && P > 0) || (!ldos_dev && P > 0) || P < 0) return fail(MALA_ERR_INVALID_ARG, "bad arguments");
    if (precision != MALA_MIXED && precision != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return mlp_forward(c, m, B_dev, P, ldos_dev, dos_sum_dev, precision, as_stream(stream));
}

int mala_integrate(mala_ctx* c, const void* ldos_dev, int64_t P, double cell_volume_, const mala_energy_grid* eg,
                   const double* dos_sum_dev, void* density_dev, double* dos_host, double* fermi_eV,
                   double* band_energy_eV, double* electron_count, double* entropy_term_eV, mala_precision precision,
                   void* stream) {
    if (!c || P < 0 || (P > 0 && !ldos_dev && !dos_sum_dev)) return fail(MALA_ERR_INVALID_ARG, "bad arguments");
    MALA_TRY(check_egrid(eg));
    if (!(cell_volume_ > 0.0)) return fail(MALA_ERR_INVALID_ARG, "cell volume must be > 0");
    if (precision != MALA_MIXED && precision != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    if (density_dev && !ldos_dev) return fail(MALA_ERR_INVALID_ARG, "density needs the LDOS");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return integrate(c, ldos_dev, P, cell_volume_, eg, dos_sum_dev, density_dev, dos_host, fermi_eV, band_energy_eV,
                     electron_count, entropy_term_eV, precision, as_stream(stream));
}

int mala_integrate_noalloc(mala_ctx* c, const void* ldos_dev, int64_t P, double cell_volume_,
                           const mala_energy_grid* eg, const double* dos_sum_dev, void* density_dev, double* dos_host,
                           double* fermi_eV, double* band_energy_eV, double* electron_count,
                           double* entropy_term_eV, mala_precision precision, void* stream) {
    if (!c || P < 0 || (P > 0 && !ldos_dev && !dos_sum_dev)) return fail(MALA_ERR_INVALID_ARG, "bad arguments");
    MALA_TRY(check_egrid(eg));
    if (!(cell_volume_ > 0.0)) return fail(MALA_ERR_INVALID_ARG, "cell volume must be > 0");
    if (precision != MALA_MIXED && precision != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    if (density_dev && !ldos_dev) return fail(MALA_ERR_INVALID_ARG, "density needs the LDOS");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return integrate_noalloc(c, ldos_dev, P, cell_volume_, eg, dos_sum_dev, density_dev, dos_host, fermi_eV,
                             band_energy_eV, electron_count, entropy_term_eV, precision, as_stream(stream));
}

int mala_electron_count(mala_ctx* c, const double* dos_host, const mala_energy_grid* eg, double mu, double* count) {
    if (!c || !dos_host || !count || !std::isfinite(mu)) return fail(MALA_ERR_INVALID_ARG, "bad arguments");
    MALA_TRY(check_egrid(eg));
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return electron_count_at(c, dos_host, eg, mu, count, c->stream);
}

int mala_predict(mala_ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, const mala_model* m,
                 const mala_energy_grid* eg, mala_precision prec, void* density_host, mala_result* res, void* stream) {
    if (!c || !res) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    memset(res, 0, sizeof(*res));
    MALA_TRY(check_path_args(snap, bp, m, eg, prec));
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    const int64_t P = (int64_t)snap->grid[0] * snap->grid[1] * snap->grid[2];
    const int nB = n_triples(bp->twojmax), nE = eg->n_E;
    const size_t e = prec == MALA_MIXED ? 4 : 8, l = prec == MALA_MIXED ? 2 : 8;
    MALA_TRY(c->ws_B.reserve(c, (size_t)P * nB * e + 256));
    MALA_TRY(c->ws_ldos.reserve(c, (size_t)P * nE * l + 256));
    MALA_TRY(c->ws_dens.reserve(c, (size_t)P * e + 256));
    MALA_TRY(c->ws_dos.reserve(c, (size_t)nE * 8 + 256));
    cudaStream_t st = as_stream(stream);
    int rc = run_path(c, snap, bp, m, eg, prec, c->ws_B.ptr, c->ws_ldos.ptr, c->ws_dens.ptr, c->ws_dos.as<double>(), res,
                      nullptr, st);
    res->dos = c->host_dos;
    if (rc != MALA_OK && rc != MALA_ERR_FERMI_BRACKET) return rc;
    if (density_host) {
        MALA_CUDA_TRY(cudaMemcpyAsync(density_host, c->ws_dens.ptr, (size_t)P * e, cudaMemcpyDeviceToHost, st));
        MALA_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return rc;
}

int mala_predict_batch(mala_ctx* c, int32_t n, const mala_snapshot* snaps, const mala_bispectrum_params* bp,
                       const mala_model* m, const mala_energy_grid* egs, mala_precision prec, void* density_host,
                       mala_result* res, void* stream) {
    if (!c || !res || !snaps || !egs) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    if (n < 1) return fail(MALA_ERR_INVALID_ARG, "need n >= 1 snapshots");
    memset(res, 0, sizeof(mala_result) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        MALA_TRY(check_path_args(&snaps[i], bp, m, &egs[i], prec));
        if (egs[i].n_E != egs[0].n_E) return fail(MALA_ERR_INVALID_ARG, "energy grids of a batch need one n_E");
    }
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    std::vector<int64_t> row(n + 1, 0);
    for (int i = 0; i < n; ++i) row[i + 1] = row[i] + (int64_t)snaps[i].grid[0] * snaps[i].grid[1] * snaps[i].grid[2];
    const int64_t P = row[n];
    const int nB = n_triples(bp->twojmax), nE = egs[0].n_E;
    const size_t e = prec == MALA_MIXED ? 4 : 8, l = prec == MALA_MIXED ? 2 : 8;
    MALA_TRY(c->ws_B.reserve(c, (size_t)P * nB * e + 256));
    MALA_TRY(c->ws_ldos.reserve(c, (size_t)P * nE * l + 256));
    MALA_TRY(c->ws_dens.reserve(c, (size_t)P * e + 256));
    cudaStream_t st = as_stream(stream);
    char* B = c->ws_B.as<char>();
    char* L = c->ws_ldos.as<char>();
    char* D = c->ws_dens.as<char>();
    c->batch_dos.assign((size_t)n * nE, 0.0);
    MALA_TRY(c->ws_dos.reserve(c, (size_t)nE * 8 + 256));
    std::vector<const mala_snapshot*> sp(n);
    std::vector<const mala_energy_grid*> ep(n);
    std::vector<double*> dh(n);
    std::vector<mala_result*> rp(n);
    for (int i = 0; i < n; ++i) {
        sp[i] = &snaps[i];
        ep[i] = &egs[i];
        dh[i] = c->batch_dos.data() + (size_t)i * nE;
        rp[i] = &res[i];
    }
    const int first_rc = run_path_batch(c, n, sp.data(), bp, m, ep.data(), prec, B, L, D, c->ws_dos.as<double>(),
                                        dh.data(), rp.data(), st);
    if (first_rc != MALA_OK && first_rc != MALA_ERR_FERMI_BRACKET) return first_rc;
    for (int i = 0; i < n; ++i) res[i].dos = dh[i];
    if (density_host) {
        MALA_CUDA_TRY(cudaMemcpyAsync(density_host, D, (size_t)P * e, cudaMemcpyDeviceToHost, st));
        MALA_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return first_rc;
}

int mala_submit(mala_ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, const mala_model* m,
                const mala_energy_grid* eg, mala_precision prec, uint64_t* ticket) {
    if (!c || !ticket) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    MALA_TRY(check_path_args(snap, bp, m, eg, prec));
    if (!c->server) {
        std::lock_guard<std::mutex> lk(c->mu);
        MALA_TRY(server_start(c));
    }
    auto r = std::make_unique<Request>();
    r->pos.assign(snap->pos, snap->pos + 3 * (size_t)snap->n_atoms);
    if (snap->species) r->species.assign(snap->species, snap->species + snap->n_atoms);
    r->snap = *snap;
    r->snap.pos = r->pos.data();
    r->snap.species = snap->species ? r->species.data() : nullptr;
    r->bp = *bp;
    if (bp->weights) {
        r->weights.assign(bp->weights, bp->weights + bp->n_species);
        r->bp.weights = r->weights.data();
    }
    r->eg = *eg;
    r->model = m;
    r->prec = prec;
    r->P = (int64_t)snap->grid[0] * snap->grid[1] * snap->grid[2];
    r->out_bytes = path_output_bytes(r->P, n_triples(bp->twojmax), eg->n_E, prec);
    r->t_submit = std::chrono::steady_clock::now();
    Server* sv = c->server;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->ticket = sv->next_ticket++;
        *ticket = r->ticket;
        sv->queue.push_back(r->ticket);
        sv->reqs[r->ticket] = std::move(r);
    }
    sv->cv_work.notify_one();
    return MALA_OK;
}

static int fill_result(Request* r, mala_result* out) {
    if (r->state != 2) return MALA_PENDING;
    if (out) *out = r->res;
    if (r->status != MALA_OK) return fail(r->status, "%s", r->error.c_str());
    return MALA_OK;
}

int mala_poll(mala_ctx* c, uint64_t ticket, mala_result* out) {
    if (!c || !c->server) return fail(MALA_ERR_NOT_FOUND, "no such ticket");
    Server* sv = c->server;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(MALA_ERR_NOT_FOUND, "no such ticket");
    return fill_result(it->second.get(), out);
}

int mala_wait(mala_ctx* c, uint64_t ticket, double timeout_s, mala_result* out) {
    if (!c || !c->server) return fail(MALA_ERR_NOT_FOUND, "no such ticket");
    Server* sv = c->server;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(MALA_ERR_NOT_FOUND, "no such ticket");
    Request* r = it->second.get();
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (r->state != 2) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != 2)
            return fail(MALA_ERR_TIMEOUT, "request %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
    }
    return fill_result(r, out);
}

int mala_release(mala_ctx* c, uint64_t ticket) {
    if (!c || !c->server) return fail(MALA_ERR_NOT_FOUND, "no such ticket");
    Server* sv = c->server;
    std::unique_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->reqs.find(ticket);
        if (it == sv->reqs.end()) return fail(MALA_ERR_NOT_FOUND, "no such ticket");
        if (it->second->state != 2) return fail(MALA_ERR_INVALID_ARG, "request %llu is still running", (unsigned long long)ticket);
        r = std::move(it->second);
        sv->reqs.erase(it);
        if (r->out && --r->out->refs == 0) {
            if (r->out->ptr) cudaFree(r->out->ptr);
            c->used -= r->out->bytes;
            sv->out_live -= r->out->bytes;
            delete r->out;
        }
        r->out = nullptr;
    }
    sv->cv_work.notify_all();
    return MALA_OK;
}

int mala_band_energy_gradient(mala_ctx* c, const double* dos_host, const mala_energy_grid* eg, double* grad_host,
                              double* fermi, double* mu_tilde, void* stream) {
    if (!c || !dos_host || !grad_host) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    MALA_TRY(check_egrid(eg));
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    cudaStream_t st = as_stream(stream);
    const int nE = eg->n_E;
    MALA_TRY(c->ws_w.reserve(c, sizeof(double) * 2 * (size_t)nE + 256));
    double* D = c->ws_w.as<double>();
    double* g = D + nE;
    MALA_CUDA_TRY(cudaMemcpyAsync(D, dos_host, sizeof(double) * nE, cudaMemcpyHostToDevice, st));
    double eF = 0.0, mt = 0.0;
    const int rc = energy_gradient(c, D, 1.0, eg, 1.0, g, &eF, &mt, st);
    if (fermi) *fermi = eF;
    if (mu_tilde) *mu_tilde = mt;
    if (rc != MALA_OK) return rc;
    MALA_CUDA_TRY(cudaMemcpyAsync(grad_host, g, sizeof(double) * nE, cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaStreamSynchronize(st));
    return MALA_OK;
}

int mala_ldos_backward(mala_ctx* c, const mala_model* m, const void* B_dev, int64_t P, const double* v_host,
                       void* beta_dev, mala_precision prec, void* stream) {
    if (!c || !m || !v_host || (P > 0 && (!B_dev || !beta_dev))) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    if (P < 0) return fail(MALA_ERR_INVALID_ARG, "P < 0");
    if (prec != MALA_MIXED && prec != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    cudaStream_t st = as_stream(stream);
    const int nE = m->dims[m->n_layers];
    MALA_TRY(c->ws_w.reserve(c, sizeof(double) * (size_t)nE + 256));
    MALA_CUDA_TRY(cudaMemcpyAsync(c->ws_w.ptr, v_host, sizeof(double) * nE, cudaMemcpyHostToDevice, st));
    MALA_TRY(mlp_backward(c, m, B_dev, P, c->ws_w.as<double>(), beta_dev, prec, st));
    MALA_CUDA_TRY(cudaStreamSynchronize(st));
    return MALA_OK;
}

int mala_descriptor_forces(mala_ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                           const void* beta_dev, double* forces_host, mala_precision prec, void* stream) {
    if (!c || !forces_host) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    MALA_TRY(check_snapshot(snap));
    MALA_TRY(check_bparams(bp));
    if (prec != MALA_MIXED && prec != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    const int64_t P = (int64_t)snap->grid[0] * snap->grid[1] * snap->grid[2];
    if (P > 0 && !beta_dev) return fail(MALA_ERR_INVALID_ARG, "beta is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    cudaStream_t st = as_stream(stream);
    NbrOut nl;
    MALA_TRY(stage_force_descriptors(c, snap, bp, prec, nullptr, &nl, st));
    return adjoint_of_staged(c, snap, bp, prec, beta_dev, nl, forces_host, st);
}

int mala_band_forces(mala_ctx* c, const mala_snapshot* snap, const mala_bispectrum_params* bp, const mala_model* m,
                     const mala_energy_grid* eg, mala_precision prec, double* forces_host, mala_result* res,
                     void* stream) {
    if (!c || !res || !forces_host) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    memset(res, 0, sizeof(*res));
    MALA_TRY(check_path_args(snap, bp, m, eg, prec));
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    cudaStream_t st = as_stream(stream);
    const int64_t P = (int64_t)snap->grid[0] * snap->grid[1] * snap->grid[2];
    const int nB = n_triples(bp->twojmax), nE = eg->n_E;
    const size_t e = prec == MALA_MIXED ? 4 : 8, l = prec == MALA_MIXED ? 2 : 8;
    MALA_TRY(c->ws_B.reserve(c, (size_t)P * nB * e + 256));
    MALA_TRY(c->ws_ldos.reserve(c, (size_t)P * nE * l + 256));
    MALA_TRY(c->ws_dens.reserve(c, (size_t)P * e + 256));
    MALA_TRY(c->ws_dos.reserve(c, (size_t)nE * 8 + 256));
    MALA_TRY(c->ws_w.reserve(c, sizeof(double) * (size_t)nE + 256));
    // forward: descriptors (with u and neighbour lists), LDOS, integrals
    NbrOut nl;
    MALA_TRY(stage_force_descriptors(c, snap, bp, prec, c->ws_B.ptr, &nl, st));
    MALA_TRY(mlp_forward(c, m, c->ws_B.ptr, P, c->ws_ldos.ptr, c->ws_dos.as<double>(), prec, st));
    double eF = 0.0, Eb = 0.0, Ne = 0.0, TS = 0.0;
    const double vol = cell_volume(snap), dV = vol / (double)(P > 0 ? P : 1);
    int rc = integrate(c, c->ws_ldos.ptr, P, vol, eg, c->ws_dos.as<double>(), c->ws_dens.ptr, nullptr, &eF, &Eb, &Ne,
                       &TS, prec, st);
    res->status = rc;
    res->n_B = nB;
    res->n_E = nE;
    res->n_points = P;
    res->fermi_eV = eF;
    res->band_energy_eV = Eb;
    res->electron_count = Ne;
    res->entropy_term_eV = TS;
    res->B_dev = c->ws_B.ptr;
    res->ldos_dev = c->ws_ldos.ptr;
    res->density_dev = c->ws_dens.ptr;
    res->dos = c->host_dos;
    if (rc != MALA_OK) return rc;
    // backward: dE_b/dLDOS = dV dE_b/dD (the same vector at every point), network, descriptors
    double mt = 0.0;
    MALA_TRY(energy_gradient(c, c->ws_dos.as<double>(), dV, eg, dV, c->ws_w.as<double>(), nullptr, &mt, st));
    MALA_TRY(c->ws_force_bt.reserve(c, (size_t)P * nB * e + 256));
    MALA_TRY(mlp_backward(c, m, c->ws_B.ptr, P, c->ws_w.as<double>(), c->ws_force_bt.ptr, prec, st));
    return adjoint_of_staged(c, snap, bp, prec, c->ws_force_bt.ptr, nl, forces_host, st);
}

int mala_ace_count(const mala_ace_params* ap, int32_t* n_desc) {
    if (!n_desc) return fail(MALA_ERR_INVALID_ARG, "NULL argument");
    MALA_TRY(check_ace_params(ap));
    *n_desc = ace_count(ap);
    return MALA_OK;
}

int mala_ace_descriptors(mala_ctx* c, const mala_snapshot* snap, const mala_ace_params* ap, void* D_dev,
                         mala_precision prec, void* stream) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    MALA_TRY(check_snapshot(snap));
    MALA_TRY(check_ace_params(ap));
    if (prec != MALA_MIXED && prec != MALA_FP64_PLAIN) return fail(MALA_ERR_INVALID_ARG, "bad precision");
    const int64_t P = (int64_t)snap->grid[0] * snap->grid[1] * snap->grid[2];
    if (P > 0 && !D_dev) return fail(MALA_ERR_INVALID_ARG, "output is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    cudaStream_t st = as_stream(stream);
    NbrOut nl;
    MALA_TRY(stage_lists_only(c, snap, ap->rcut, ap->n_species, &nl, st));
    const SnapDev& sd = static_cast<const BatchSnap*>(c->host_batch)[0].sd;
    return ace_from_lists(c, sd, snap, ap, nl, D_dev, prec, st);
}

}  // extern "C"
