// Request server: a persistent pool of worker threads, each with its own CUDA stream,
// serving (structure, frequencies, field directions) solve requests as they arrive.
//
//   - Structures stay resident: requests reference geometries built once with
//     wfq_build_geometry (D, Kbar, atom data stay on the device between requests).
//   - Admission by device-memory footprint: a batch starts only while the device bytes of
//     the structures with requests queued or running, the footprints of the batches in
//     flight and its own footprint stay within the server's budget.
//   - Continuous batching: when a worker becomes free it takes the oldest admissible
//     request and merges into the same block solve every queued request on the same
//     structure with the same solver settings (the columns of all of them share D and
//     Kbar), up to a column limit.  Requests that arrive while others run are picked up
//     as soon as a worker and memory free up; batches on different streams overlap on
//     the device.
//   - Solver of a batch: shifted GMRES when the structure has a stored D (one real
//     Arnoldi process per distinct field direction serves every frequency of every merged
//     request), else mixed block GMRES(m) with FP64 refinement.
//   - Each request's result (its columns of q, its per-column statistics) is written to
//     the caller's host buffers; submit / completion times give its latency.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    wfq_geom *g = nullptr;
    std::vector<double> omega;   // nfreq
    std::vector<double> dirs;    // ndir x 3
    int ndir = 0;
    double E0 = 1.0;
    int m = 50;
    double rel_tol = 1e-8;
    int max_iter = 1000;
    double *q_host = nullptr;        // n x ncols complex128 (caller-owned)
    wfq_stats *stats = nullptr;      // ncols (caller-owned, may be null)
    int64_t ncols() const { return (int64_t)omega.size() * ndir; }
    clk::time_point t_submit, t_start, t_done;
    int status = WFQ_OK;
    bool done = false;
    int batch_columns = 0;
};

// Structures with a stored D (FP32 pair planes or FP64) are served by shifted GMRES; the
// others by mixed block GMRES(m).
bool use_shifted(const wfq_geom *g) { return g->Dfh != nullptr || g->D64 != nullptr; }

// Distinct field directions of a batch (exact comparison) and, per request, the index of
// each of its directions in that list.
int unique_dirs(const std::vector<Request *> &batch, std::vector<double> &dirs, std::vector<std::vector<int>> &map) {
    dirs.clear();
    map.assign(batch.size(), {});
    for (size_t k = 0; k < batch.size(); ++k) {
        const Request *r = batch[k];
        for (int d = 0; d < r->ndir; ++d) {
            const double *v = &r->dirs[3 * (size_t)d];
            int found = -1;
            for (size_t u = 0; u < dirs.size() / 3 && found < 0; ++u)
                if (dirs[3 * u] == v[0] && dirs[3 * u + 1] == v[1] && dirs[3 * u + 2] == v[2]) found = (int)u;
            if (found < 0) {
                found = (int)(dirs.size() / 3);
                dirs.insert(dirs.end(), v, v + 3);
            }
            map[k].push_back(found);
        }
    }
    return (int)(dirs.size() / 3);
}

bool same_settings(const Request *a, const Request *b) {
    return a->g == b->g && a->E0 == b->E0 && a->m == b->m && a->rel_tol == b->rel_tol &&
           a->max_iter == b->max_iter;
}

// columns [c0, c0 + nc) of the n x ncol block src -> dst (n x nc)
__global__ void k_take_cols(uint32_t total, uint32_t nc, int64_t ncol, int64_t c0, const double2 *__restrict__ src,
                            double2 *__restrict__ dst) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t r = e / nc, k = e % nc;
    dst[e] = src[(int64_t)r * ncol + c0 + k];
}

}  // namespace

struct wfq_server {
    wfq_ctx *ctx = nullptr;
    size_t budget = 0;
    size_t in_use = 0;      // footprints of the batches in flight
    size_t resident = 0;    // device bytes of the structures with requests queued or running
    std::unordered_map<const wfq_geom *, int64_t> refs;   // requests queued or running per structure
    int64_t max_cols = 384;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<int64_t, Request *> reqs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    bool stop = false;
    int64_t next_id = 1;
    int64_t batches = 0, merged = 0;

    // Structure accounting (under the lock): a structure's bytes count against the budget
    // while it has requests queued or running.
    void hold(const wfq_geom *g) {
        if (refs[g]++ == 0) resident += g->bytes;
    }
    void release(const wfq_geom *g) {
        auto it = refs.find(g);
        if (it != refs.end() && --it->second == 0) {
            resident -= g->bytes;
            refs.erase(it);
        }
    }

    // Pops a batch (under the lock).  Returns false when the server is stopping and the
    // queue is empty.
    bool next_batch(std::unique_lock<std::mutex> &lk, std::vector<Request *> &batch, size_t &fp) {
        for (;;) {
            if (stop && queue.empty()) return false;
            if (!queue.empty()) {
                Request *head = queue.front();
                int64_t cols = head->ncols();
                std::vector<size_t> pick{0};
                for (size_t i = 1; i < queue.size(); ++i) {
                    Request *r = queue[i];
                    if (same_settings(head, r) && cols + r->ncols() <= max_cols) {
                        pick.push_back(i);
                        cols += r->ncols();
                    }
                }
                size_t need;
                if (use_shifted(head->g)) {
                    std::vector<Request *> pb;
                    for (size_t i : pick) pb.push_back(queue[i]);
                    std::vector<double> ud;
                    std::vector<std::vector<int>> um;
                    need = wfq::shifted_footprint(head->g, cols, unique_dirs(pb, ud, um), 0);
                } else {
                    need = wfq::solve_footprint(head->g, cols, head->m, WFQ_PREC_MIXED);
                }
                if (in_use == 0 || in_use + need + resident <= budget) {
                    batch.clear();
                    for (size_t k = pick.size(); k-- > 0;) {
                        batch.insert(batch.begin(), queue[pick[k]]);
                        queue.erase(queue.begin() + (std::ptrdiff_t)pick[k]);
                    }
                    in_use += need;
                    fp = need;
                    return true;
                }
            }
            cv_work.wait(lk);
        }
    }

    void run(int w) {
        cudaSetDevice(ctx->device);
        cudaGetLastError();
        cudaStream_t s = streams[w];
        for (;;) {
            std::vector<Request *> batch;
            size_t fp = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (!next_batch(lk, batch, fp)) return;
                ++batches;
                merged += (int64_t)batch.size() - 1;
            }
            const auto t0 = clk::now();
            for (Request *r : batch) r->t_start = t0;
            solve_batch(batch, s);
            const auto t1 = clk::now();
            {
                std::lock_guard<std::mutex> lk(mu);
                in_use -= fp;
                for (Request *r : batch) {
                    r->t_done = t1;
                    r->done = true;
                    release(r->g);
                }
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }

    void solve_batch(std::vector<Request *> &batch, cudaStream_t s) {
        using namespace wfq;
        Request *head = batch.front();
        wfq_geom *g = head->g;
        // merged column list: each request keeps its own (omega x dirs) columns in order;
        // directions shared by several requests are one direction of the batch
        std::vector<double> col_om, dirs;
        std::vector<int> col_dir;
        std::vector<int64_t> first_col;
        std::vector<std::vector<int>> dmap;
        const int ndir_u = unique_dirs(batch, dirs, dmap);
        for (size_t k = 0; k < batch.size(); ++k) {
            Request *r = batch[k];
            first_col.push_back((int64_t)col_om.size());
            for (double om : r->omega)
                for (int d = 0; d < r->ndir; ++d) {
                    col_om.push_back(om);
                    col_dir.push_back(dmap[k][d]);
                }
            r->batch_columns = 0;
        }
        const int64_t cc = (int64_t)col_om.size(), n = g->n;
        for (Request *r : batch) r->batch_columns = (int)cc;
        int rc = WFQ_OK;
        DevBuf<double2> q, part;
        std::vector<wfq_stats> st(cc);
        if ((rc = q.alloc(g->ctx, (size_t)n * cc, s)) == WFQ_OK) {
            SolveArgs a;
            a.ndir = ndir_u;
            a.dirs = dirs.data();
            a.col_omega = col_om.data();
            a.col_dir = col_dir.data();
            a.ncols = cc;
            a.E0 = head->E0;
            a.m = head->m;
            a.rel_tol = head->rel_tol;
            a.max_iter = head->max_iter;
            // continuations of a BEM batch run in FP64 unless its bf16 planes are stored
            // (its operator is never regenerated from the coordinates)
            a.prec = (g->op == OP_BEM && !g->Dhi) ? WFQ_PREC_FP64 : WFQ_PREC_MIXED;
            a.q = q.ptr;
            a.stats = st.data();
            if (use_shifted(g)) {
                a.m = 0;   // basis cap: the solver's default; continuations run GMRES(50)
                rc = solve_gmres_shifted(g, a, s);
            } else {
                rc = solve_gmres(g, a, s);
            }
        }
        for (size_t k = 0; k < batch.size(); ++k) {
            Request *r = batch[k];
            const int64_t nc = r->ncols();
            int rrc = (rc == WFQ_OK || rc == WFQ_ENOCONV) ? WFQ_OK : rc;
            if (rrc == WFQ_OK) {
                bool all_ok = true;
                for (int64_t c = 0; c < nc; ++c) {
                    if (r->stats) r->stats[c] = st[first_col[k] + c];
                    all_ok = all_ok && st[first_col[k] + c].status == WFQ_OK;
                }
                rrc = all_ok ? WFQ_OK : WFQ_ENOCONV;
                if (r->q_host) {
                    if (part.ptr == nullptr && part.alloc(g->ctx, (size_t)n * cc, s) != WFQ_OK) {
                        rrc = WFQ_ENOMEM;
                    } else {
                        const uint32_t tot = (uint32_t)(n * nc);
                        k_take_cols<<<(tot + 255) / 256, 256, 0, s>>>(tot, (uint32_t)nc, cc, first_col[k], q.ptr,
                                                                       part.ptr);
                        note_launch();
                        if (cudaMemcpyAsync(r->q_host, part.ptr, sizeof(double2) * n * nc, cudaMemcpyDeviceToHost, s) !=
                                cudaSuccess ||
                            cudaStreamSynchronize(s) != cudaSuccess) {
                            cudaGetLastError();
                            rrc = WFQ_ECUDA;
                        }
                    }
                }
            }
            r->status = rrc;
        }
        cudaStreamSynchronize(s);
    }
};

using namespace wfq;

extern "C" {

int wfq_server_create(wfq_ctx *ctx, int nworkers, int64_t budget_bytes, int max_columns, wfq_server **out) {
    if (!ctx || !out) return fail(WFQ_EINVAL, "NULL argument");
    if (nworkers < 1 || nworkers > 64 || budget_bytes < 1 || max_columns < 1)
        return fail(WFQ_EINVAL, "nworkers in 1..64, budget and max_columns > 0");
    *out = nullptr;
    cudaSetDevice(ctx->device);
    auto *sv = new wfq_server;
    sv->ctx = ctx;
    sv->budget = (size_t)budget_bytes;
    sv->max_cols = max_columns;
    for (int w = 0; w < nworkers; ++w) {
        cudaStream_t s = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
            delete sv;
            return fail(WFQ_ECUDA, std::string("server stream: ") + cudaGetErrorString(e));
        }
        sv->streams.push_back(s);
    }
    for (int w = 0; w < nworkers; ++w) sv->workers.emplace_back([sv, w] { sv->run(w); });
    *out = sv;
    return WFQ_OK;
}

int wfq_server_submit(wfq_server *sv, wfq_geom *g, int64_t nfreq, const double *omega, int ndir, const double *dirs,
                      double E0, int m, double rel_tol, int max_iter, double *q_host, wfq_stats *stats,
                      int64_t *request_id) {
    if (!sv || !g || !omega || !dirs || !request_id) return fail(WFQ_EINVAL, "NULL argument");
    if (nfreq < 1 || ndir < 1 || m < 1 || max_iter < 1 || !(rel_tol > 0.0 && rel_tol < 1.0) || E0 == 0.0)
        return fail(WFQ_EINVAL, "bad request shape or settings");
    for (int64_t f = 0; f < nfreq; ++f) {
        if (!std::isfinite(omega[f])) return fail(WFQ_EINVAL, "non-finite omega");
        if (omega[f] == 0.0) return fail(WFQ_ESINGULAR, "omega = 0: z(0) = 0 and A is singular");
    }
    if (g->op == OP_BEM) {
        const ShiftModel zm = shift_model(g);
        for (int64_t f = 0; f < nfreq; ++f) {
            const double2 z = z_eval(zm, omega[f]);
            if (!(std::isfinite(z.x) && std::isfinite(z.y)))
                return fail(WFQ_EINVAL, "eps_in(omega) = eps_out: Lambda(omega) is infinite");
        }
    }
    if (g->ctx != sv->ctx) return fail(WFQ_EINVAL, "geometry belongs to another context");
    const int64_t cols = nfreq * ndir;
    if (cols > sv->max_cols) return fail(WFQ_EINVAL, "request has more columns than the server's batch limit");
    const size_t need = use_shifted(g) ? shifted_footprint(g, cols, ndir, 0) : solve_footprint(g, cols, m, WFQ_PREC_MIXED);
    if (need + g->bytes > sv->budget)
        return fail(WFQ_ENOMEM, "the structure's device bytes plus the request's footprint exceed the server's "
                                "memory budget");
    auto *r = new Request;
    r->g = g;
    r->omega.assign(omega, omega + nfreq);
    r->dirs.assign(dirs, dirs + 3 * ndir);
    r->ndir = ndir;
    r->E0 = E0;
    r->m = m;
    r->rel_tol = rel_tol;
    r->max_iter = max_iter;
    r->q_host = q_host;
    r->stats = stats;
    r->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete r;
            return fail(WFQ_EINVAL, "server is shutting down");
        }
        r->id = sv->next_id++;
        sv->reqs[r->id] = r;
        sv->queue.push_back(r);
        sv->hold(g);
        *request_id = r->id;
    }
    sv->cv_work.notify_one();
    return WFQ_OK;
}

int wfq_server_poll(wfq_server *sv, int64_t request_id, int wait, int *done, int *status, double *latency_s,
                    double *queue_s, int *batch_columns) {
    if (!sv) return fail(WFQ_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(request_id);
    if (it == sv->reqs.end()) return fail(WFQ_EINVAL, "unknown request id");
    Request *r = it->second;
    if (wait) sv->cv_done.wait(lk, [r] { return r->done; });
    if (done) *done = r->done ? 1 : 0;
    if (r->done) {
        if (status) *status = r->status;
        if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
        if (queue_s) *queue_s = std::chrono::duration<double>(r->t_start - r->t_submit).count();
        if (batch_columns) *batch_columns = r->batch_columns;
        sv->reqs.erase(it);
        delete r;
    }
    return WFQ_OK;
}

int wfq_server_destroy(wfq_server *sv) {
    if (!sv) return WFQ_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    for (auto &kv : sv->reqs) delete kv.second;
    delete sv;
    return WFQ_OK;
}

}  // extern "C"
