// Batched and served LM steps: many independent systems sharing one GPU.
//
// Both engines run each instance's step (build, IRL, refinement) as the same
// sequence of kernels that lm_build_OG + irl_step issue for it alone, on one
// stream of a pool, and advance instances from the host as their device work
// completes (event queries, no device-wide synchronisation). Instances on
// different streams overlap on the device: the small pencils of mid-sized
// systems leave most SMs idle when run one after another, and their builds,
// products and Lanczos steps fill each other's gaps when run together.
//
// The pencil-product grid of every new pencil shape can be autotuned: each
// candidate grid (one CTA per SM, 1/2, 1/4, 1/8 of that) is timed alone on the
// built pencil. Under concurrency a product holds two shared resources for its
// duration t: a share g/SMs of the SMs and a share of the HBM bandwidth, at
// least (bytes streamed / streaming rate) / t. Its cost is the larger share
// times t, max(t g / SMs, bytes / rate); the grid of least cost is kept, and
// among grids within 3 % of it the fastest. A product that streams from HBM
// costs about the same on any grid (fewer SMs only stretch it), so it keeps a
// large grid and its latency; a small, cache-resident one moves to a small
// grid and leaves the other SMs to other instances.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace {

// Pencils of the engines replay captured IRL cycles (irl.cu) unless
// IRLNQS_CYCLE_GRAPHS=0 (for timing the launch path against them).
int cycle_graphs_on() {
    const char *e = getenv("IRLNQS_CYCLE_GRAPHS");
    return !(e && e[0] == '0');
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

using GridKey = std::tuple<int, int64_t, int, int>;  // ldp, rows, storage, symmetrisation

// Pick (once per shape) the pencil grid of least cost (rule above).
int autotune_grid(lm_pencil *p, cudaStream_t s, std::map<GridKey, int> &cache) {
    lm_ctx *ctx = p->ctx;
    const GridKey key{p->ldp, p->n_rows, p->prec, p->sym};
    auto it = cache.find(key);
    if (it != cache.end()) {
        p->g_pencil = it->second;
        return LM_OK;
    }
    const int prec = p->prec == LM_FP64 ? LM_FP64 : p->prec;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return lm_fail(ctx, LM_ERR_CUDA, "cudaEventCreate");
    cudaMemsetAsync(p->tvec, 0, p->ldp * sizeof(double), s);
    const int prof = ctx->profile;
    ctx->profile = 0;  // keep the tuning launches out of the counters
    // bytes one product streams: both factors and the weights
    const int esize = p->prec == LM_FP32 ? 4 : p->prec == LM_BF16 ? 2 : 8;
    const double bytes = (double)p->n_rows * ((double)p->ldp * esize * 2 + 8);
    const double hbm_ms = ctx->hbm_bytes_per_ms > 0 ? bytes / ctx->hbm_bytes_per_ms : 0.0;
    int grid[4], n = 0;
    double t[4], cost[4];
    int rc = LM_OK;
    for (int div : {1, 2, 4, 8}) {
        const int g = ctx->sms / div;
        if (g < 4 || (div > 1 && (int64_t)g * 8 > p->n_rows)) continue;
        p->g_pencil = g;
        rc = lm_launch_pencil(p, p->tvec, p->sym, prec, 0, nullptr, s);
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && !rc; ++r) rc = lm_launch_pencil(p, p->tvec, p->sym, prec, 0, nullptr, s);
        cudaEventRecord(e1, s);
        if (!rc) rc = lm_cuda_check(ctx, cudaEventSynchronize(e1), "grid autotuning");
        if (rc) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        grid[n] = g;
        t[n] = ms / 3.0;
        cost[n] = std::max(t[n] * g / ctx->sms, hbm_ms);
        ++n;
    }
    ctx->profile = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int best = ctx->sms;
    if (n > 0) {
        double least = cost[0];
        for (int i = 1; i < n; ++i) least = std::min(least, cost[i]);
        int b = -1;
        for (int i = 0; i < n; ++i)
            if (cost[i] <= 1.03 * least && (b < 0 || t[i] < t[b])) b = i;
        best = grid[b];
    }
    p->g_pencil = best;
    if (!rc) cache[key] = best;
    return rc;
}

bool event_done(cudaEvent_t e) {
    const cudaError_t q = cudaEventQuery(e);
    if (q == cudaErrorNotReady) return false;
    return true;  // completed, or an error that the next CUDA check reports
}

}  // namespace

// ---------------------------------------------------------------- batch
struct lm_batch {
    lm_ctx *ctx;
    std::vector<cudaStream_t> streams;
    cudaStream_t tune;  // grid tuning runs alone on this stream
    int autotune;
    std::vector<lm_pencil *> pencils;  // per item index, kept across runs
    std::map<GridKey, int> grids;
};

extern "C" int lm_batch_create(lm_ctx *ctx, int n_streams, int autotune, lm_batch **out) {
    if (!ctx || !out) return LM_ERR_ARG;
    if (n_streams < 1 || n_streams > 64) return lm_fail(ctx, LM_ERR_ARG, "1..64 streams");
    cudaSetDevice(ctx->device);
    lm_batch *b = new lm_batch();
    b->ctx = ctx;
    b->autotune = autotune;
    if (cudaStreamCreateWithFlags(&b->tune, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return lm_fail(ctx, LM_ERR_CUDA, "cudaStreamCreate");
    }
    for (int i = 0; i < n_streams; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t t : b->streams) cudaStreamDestroy(t);
            cudaStreamDestroy(b->tune);
            delete b;
            return lm_fail(ctx, LM_ERR_CUDA, "cudaStreamCreate");
        }
        b->streams.push_back(s);
    }
    *out = b;
    return LM_OK;
}

extern "C" int lm_batch_run(lm_batch *b, int n, const lm_batch_item *items, irl_result *results,
                            int *grid_out) {
    if (!b || n < 0 || (n > 0 && (!items || !results))) return LM_ERR_ARG;
    lm_ctx *ctx = b->ctx;
    cudaSetDevice(ctx->device);
    enum { I_BUILD, I_IRL, I_DONE };
    struct Inst {
        int state = I_BUILD;
        IrlJob *job = nullptr;
        cudaEvent_t ev = nullptr;
        cudaStream_t s = nullptr;
        int rc = LM_OK;
        bool fresh = false;
    };
    if ((int)b->pencils.size() < n) b->pencils.resize(n, nullptr);
    std::vector<Inst> in(n);
    int first_rc = LM_OK;
    auto fail = [&](Inst &I, int rc) {
        I.rc = rc;
        I.state = I_DONE;
        if (!first_rc) first_rc = rc;
    };
    for (int i = 0; i < n; ++i) {
        Inst &I = in[i];
        I.s = b->streams[i % b->streams.size()];
        cudaEventCreateWithFlags(&I.ev, cudaEventDisableTiming);
        const lm_batch_item &it = items[i];
        lm_pencil *&p = b->pencils[i];
        if (p && (p->n != it.sys.n_orb || p->na != it.sys.n_alpha || p->nb != it.sys.n_beta ||
                  p->nh != it.sys.n_hidden || p->prec != it.precision ||
                  (it.rows && p->n_rows != it.n_rows))) {
            cudaDeviceSynchronize();
            lm_pencil_release(p);
            p = nullptr;
        }
        I.fresh = p == nullptr;
        int rc = lm_build_enqueue(ctx, &it.sys, it.theta, it.rows, it.weights, it.n_rows,
                                  (lm_precision)it.precision, I.s, &p);
        if (!rc) p->cycle_graphs = cycle_graphs_on();
        if (!rc) rc = lm_cuda_check(ctx, cudaEventRecord(I.ev, I.s), "event");
        if (rc) fail(I, rc);
    }
    for (int active = n; active > 0;) {
        active = 0;
        bool progress = false;
        for (int i = 0; i < n; ++i) {
            Inst &I = in[i];
            if (I.state == I_DONE) continue;
            ++active;
            int rc = LM_OK;
            if (I.state == I_BUILD) {
                if (!event_done(I.ev)) continue;
                progress = true;
                rc = lm_cuda_check(ctx, cudaEventSynchronize(I.ev), "build");
                lm_pencil *p = b->pencils[i];
                if (!rc) rc = lm_build_finish(p);
                // a new pencil shape: tune its product grid (a few launches) first
                if (!rc && I.fresh && b->autotune) rc = autotune_grid(p, b->tune, b->grids);
                if (!rc)
                    rc = irl_job_create(p, &items[i].irl, nullptr, items[i].dtheta_out,
                                        items[i].theta_inout, I.s, &I.job);
                int done = 0;
                if (!rc) rc = irl_job_advance(I.job, &done);
                I.state = I_IRL;
            } else {
                if (!event_done(irl_job_event(I.job))) continue;
                progress = true;
                rc = lm_cuda_check(ctx, cudaEventSynchronize(irl_job_event(I.job)), "IRL");
                int done = 0;
                if (!rc) rc = irl_job_advance(I.job, &done);
                if (!rc && done) {
                    irl_job_result(I.job, &results[i]);
                    I.state = I_DONE;
                }
            }
            if (rc) fail(I, rc);
        }
        if (!progress && active) std::this_thread::yield();
    }
    for (int i = 0; i < n; ++i) {
        if (in[i].job) irl_job_free(in[i].job);
        if (in[i].ev) cudaEventDestroy(in[i].ev);
        if (grid_out) grid_out[i] = b->pencils[i] ? b->pencils[i]->g_pencil : 0;
    }
    return first_rc;
}

extern "C" int lm_batch_free(lm_batch *b) {
    if (!b) return LM_ERR_ARG;
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    for (lm_pencil *p : b->pencils)
        if (p) lm_pencil_release(p);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    cudaStreamDestroy(b->tune);
    delete b;
    return LM_OK;
}

// ---------------------------------------------------------------- server
namespace {

struct SysRec {
    lm_system sys;
    std::vector<double> h, eri;
    std::vector<uint64_t> rows;
    std::vector<double> weights;
    int64_t n_rows;
    int prec;
    int n_params;
    size_t footprint;
    lm_pencil *p = nullptr;
    bool busy = false;
    double last_used = 0.0;
};

struct Req {
    int64_t ticket;
    int sys_id;
    std::vector<double> theta;
    irl_params prm;
    double *dtheta_out;
    double t_submit, t_admit = 0.0;
    int state = 0;  // 0 queued, 1 building, 2 IRL
    int stream = -1;
    IrlJob *job = nullptr;
    cudaEvent_t ev = nullptr;
    bool fresh = false;  // its build created the system's pencil
};

}  // namespace

struct lm_server {
    lm_ctx *ctx;
    cudaStream_t tune = nullptr;  // grid tuning runs alone on this stream
    // streams [0, n_high) have the device's highest priority and serve small
    // systems, the rest the lowest priority and large ones (when both pools
    // have free streams; otherwise any free stream)
    int n_high = 0;
    size_t budget, resident = 0;
    int autotune;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::vector<SysRec> systems;
    std::deque<Req *> queued;
    std::vector<Req *> inflight;
    std::deque<lm_response> finished;
    int64_t next_ticket = 1;
    std::map<GridKey, int> grids;
};

extern "C" int lm_server_create(lm_ctx *ctx, size_t hbm_budget_bytes, int n_streams, int autotune,
                                lm_server **out) {
    if (!ctx || !out) return LM_ERR_ARG;
    if (n_streams < 1 || n_streams > 64) return lm_fail(ctx, LM_ERR_ARG, "1..64 streams");
    cudaSetDevice(ctx->device);
    lm_server *v = new lm_server();
    v->ctx = ctx;
    v->budget = hbm_budget_bytes;
    v->autotune = autotune;
    if (cudaStreamCreateWithFlags(&v->tune, cudaStreamNonBlocking) != cudaSuccess) {
        delete v;
        return lm_fail(ctx, LM_ERR_CUDA, "cudaStreamCreate");
    }
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    v->n_high = std::max(1, n_streams / 2);
    for (int i = 0; i < n_streams; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, i < v->n_high ? hi : lo) !=
            cudaSuccess) {
            for (cudaStream_t t : v->streams) cudaStreamDestroy(t);
            cudaStreamDestroy(v->tune);
            delete v;
            return lm_fail(ctx, LM_ERR_CUDA, "cudaStreamCreate");
        }
        v->streams.push_back(s);
        v->stream_busy.push_back(false);
    }
    *out = v;
    return LM_OK;
}

extern "C" int lm_server_add_system(lm_server *v, const lm_system *sys, const uint64_t *rows,
                                    const double *weights, int64_t n_rows, int precision,
                                    int *system_id) {
    if (!v || !sys || !system_id || !sys->h || !sys->eri) return LM_ERR_ARG;
    if (lm_is_device_ptr(sys->h) || lm_is_device_ptr(sys->eri) ||
        (rows && lm_is_device_ptr(rows)) || (weights && lm_is_device_ptr(weights)))
        return lm_fail(v->ctx, LM_ERR_ARG, "server systems take host arrays");
    if (precision < LM_FP64 || precision > LM_DF64) return lm_fail(v->ctx, LM_ERR_ARG, "precision");
    SysRec r;
    const int n = sys->n_orb;
    r.sys = *sys;
    r.h.assign(sys->h, sys->h + (size_t)n * n);
    r.eri.assign(sys->eri, sys->eri + (size_t)n * n * n * n);
    r.sys.h = nullptr;
    r.sys.eri = nullptr;
    if (rows) r.rows.assign(rows, rows + n_rows);
    if (weights) r.weights.assign(weights, weights + n_rows);
    r.n_rows = rows ? n_rows : 0;
    r.prec = precision;
    r.n_params = (sys->n_hidden + 1) * (2 * n + 1) - 1;
    int64_t nr = n_rows;
    if (!rows) {
        auto binom = [](int a, int k) {
            double c = 1;
            for (int i = 0; i < k; ++i) c = c * (a - i) / (i + 1);
            return (int64_t)(c + 0.5);
        };
        nr = binom(n, sys->n_alpha) * binom(n, sys->n_beta);
    }
    r.footprint = lm_pencil_footprint(v->ctx, n, sys->n_hidden, nr, precision);
    if (r.footprint > v->budget)
        return lm_fail(v->ctx, LM_ERR_SIZE, "system needs %zu bytes, above the budget %zu",
                       r.footprint, v->budget);
    v->systems.push_back(std::move(r));
    *system_id = (int)v->systems.size() - 1;
    return LM_OK;
}

extern "C" int lm_server_submit(lm_server *v, int system_id, const double *theta,
                                const irl_params *prm, double *dtheta_out, int64_t *ticket) {
    if (!v || !theta || !prm || !ticket) return LM_ERR_ARG;
    if (system_id < 0 || system_id >= (int)v->systems.size())
        return lm_fail(v->ctx, LM_ERR_ARG, "unknown system %d", system_id);
    const SysRec &r = v->systems[system_id];
    Req *q = new Req();
    q->ticket = v->next_ticket++;
    q->sys_id = system_id;
    q->theta.assign(theta, theta + r.n_params);
    q->prm = *prm;
    q->prm.v0 = nullptr;
    q->dtheta_out = dtheta_out;
    q->t_submit = now_ms();
    v->queued.push_back(q);
    *ticket = q->ticket;
    return LM_OK;
}

namespace {

void server_finish(lm_server *v, Req *q, int status, const irl_result *res) {
    lm_response o;
    std::memset(&o, 0, sizeof(o));
    o.ticket = q->ticket;
    o.system_id = q->sys_id;
    o.status = status;
    const SysRec &rs = v->systems[q->sys_id];
    o.grid = rs.p ? rs.p->g_pencil : 0;
    if (res) o.result = *res;
    o.t_submit_ms = q->t_submit;
    o.t_admit_ms = q->t_admit;
    o.t_done_ms = now_ms();
    v->finished.push_back(o);
    SysRec &r = v->systems[q->sys_id];
    r.busy = false;
    r.last_used = o.t_done_ms;
    if (q->stream >= 0) v->stream_busy[q->stream] = false;
    if (q->job) irl_job_free(q->job);
    if (q->ev) cudaEventDestroy(q->ev);
    delete q;
}

// Make room for `need` bytes by evicting idle resident systems, least recently
// used first. Returns false if the budget cannot hold them.
bool server_make_room(lm_server *v, size_t need) {
    while (v->resident + need > v->budget) {
        int victim = -1;
        for (int i = 0; i < (int)v->systems.size(); ++i) {
            const SysRec &r = v->systems[i];
            if (r.p && !r.busy && (victim < 0 || r.last_used < v->systems[victim].last_used))
                victim = i;
        }
        if (victim < 0) return false;
        SysRec &r = v->systems[victim];
        lm_pencil_release(r.p);  // idle: none of its work is in flight
        r.p = nullptr;
        v->resident -= r.footprint;
    }
    return true;
}

// Start a queued request on a free stream: the build, then its IRL.
int server_admit(lm_server *v, Req *q, int stream) {
    SysRec &r = v->systems[q->sys_id];
    lm_ctx *ctx = v->ctx;
    cudaStream_t s = v->streams[stream];
    lm_system sys = r.sys;
    sys.h = r.h.data();
    sys.eri = r.eri.data();
    const bool fresh = r.p == nullptr;
    if (fresh) v->resident += r.footprint;
    int rc = lm_build_enqueue(ctx, &sys, q->theta.data(), r.rows.empty() ? nullptr : r.rows.data(),
                              r.weights.empty() ? nullptr : r.weights.data(), r.n_rows,
                              (lm_precision)r.prec, s, &r.p);
    if (rc && fresh && !r.p) v->resident -= r.footprint;
    if (!rc) r.p->cycle_graphs = cycle_graphs_on();
    q->stream = stream;
    v->stream_busy[stream] = true;
    r.busy = true;
    q->t_admit = now_ms();
    if (rc) return rc;
    q->fresh = fresh;
    cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
    q->state = 1;
    return lm_cuda_check(ctx, cudaEventRecord(q->ev, s), "event");
}

}  // namespace

extern "C" int lm_server_poll(lm_server *v, lm_response *out, int cap, int *n_out) {
    if (!v || !n_out || (cap > 0 && !out)) return LM_ERR_ARG;
    lm_ctx *ctx = v->ctx;
    cudaSetDevice(ctx->device);
    // advance the requests in flight
    for (size_t i = 0; i < v->inflight.size();) {
        Req *q = v->inflight[i];
        int rc = LM_OK;
        bool finished = false;
        if (q->state == 1) {
            if (!event_done(q->ev)) {
                ++i;
                continue;
            }
            rc = lm_cuda_check(ctx, cudaEventSynchronize(q->ev), "build");
            SysRec &r = v->systems[q->sys_id];
            if (!rc) rc = lm_build_finish(r.p);
            if (!rc && q->fresh && v->autotune)
                rc = autotune_grid(r.p, v->tune, v->grids);
            if (!rc)
                rc = irl_job_create(r.p, &q->prm, nullptr, q->dtheta_out, nullptr,
                                    v->streams[q->stream], &q->job);
            int done = 0;
            if (!rc) rc = irl_job_advance(q->job, &done);
            q->state = 2;
        } else {
            if (!event_done(irl_job_event(q->job))) {
                ++i;
                continue;
            }
            rc = lm_cuda_check(ctx, cudaEventSynchronize(irl_job_event(q->job)), "IRL");
            int done = 0;
            if (!rc) rc = irl_job_advance(q->job, &done);
            if (!rc && done) {
                irl_result res;
                irl_job_result(q->job, &res);
                server_finish(v, q, LM_OK, &res);
                finished = true;
            }
        }
        if (rc && !finished) {
            server_finish(v, q, rc, nullptr);
            finished = true;
        }
        if (finished) {
            v->inflight.erase(v->inflight.begin() + i);
        } else {
            ++i;
        }
    }
    // admit queued requests, oldest first, that have an idle system, a free
    // stream and room in the budget (later requests may pass a blocked one)
    for (auto it = v->queued.begin(); it != v->queued.end();) {
        Req *q = *it;
        SysRec &r = v->systems[q->sys_id];
        // small systems (under 64 MB of O/G) prefer the high-priority pool
        const bool small = r.footprint < ((size_t)64 << 20);
        int stream = -1;
        const int ns = (int)v->streams.size();
        for (int pass = 0; pass < 2 && stream < 0; ++pass)
            for (int k = 0; k < ns; ++k) {
                const bool high = k < v->n_high;
                if (!v->stream_busy[k] && (pass == 1 || high == small)) {
                    stream = k;
                    break;
                }
            }
        if (stream < 0) break;
        if (r.busy || (!r.p && !server_make_room(v, r.footprint))) {
            ++it;
            continue;
        }
        it = v->queued.erase(it);
        const int rc = server_admit(v, q, stream);
        if (rc) {
            server_finish(v, q, rc, nullptr);
        } else {
            v->inflight.push_back(q);
        }
    }
    int n = 0;
    while (n < cap && !v->finished.empty()) {
        out[n++] = v->finished.front();
        v->finished.pop_front();
    }
    *n_out = n;
    return LM_OK;
}

extern "C" int lm_server_pending(lm_server *v, int *n) {
    if (!v || !n) return LM_ERR_ARG;
    *n = (int)(v->queued.size() + v->inflight.size() + v->finished.size());
    return LM_OK;
}

extern "C" int lm_server_free(lm_server *v) {
    if (!v) return LM_ERR_ARG;
    cudaSetDevice(v->ctx->device);
    cudaDeviceSynchronize();
    for (Req *q : v->inflight) {
        if (q->job) irl_job_free(q->job);
        if (q->ev) cudaEventDestroy(q->ev);
        delete q;
    }
    for (Req *q : v->queued) delete q;
    for (SysRec &r : v->systems)
        if (r.p) lm_pencil_release(r.p);
    for (cudaStream_t s : v->streams) cudaStreamDestroy(s);
    cudaStreamDestroy(v->tune);
    delete v;
    return LM_OK;
}
