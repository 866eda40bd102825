// Serving runtime (fsg_server_*): a worker thread admits graph-build requests
// by slot and HBM budget, runs each on its slot's stream (requests overlap on
// the device), allocates from a private stream-ordered pool (no device-wide
// synchronization when requests come and go), and retires them in two stages:
// (1) graph built and its edge count on the host, (2) the edges on the host.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "fsg_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Pending {
    uint64_t id;
    fsg_request req;
    Clock::time_point t_submit;
    size_t bytes;
    double est_ms;  // run-time estimate for the response-ratio order
};

struct Slot {
    int state = 0;  // 0 idle, 1 building (waiting for ev_built), 2 copying edges (waiting for ev_done)
    cudaStream_t stream = nullptr;   // the admitted request's stream: stream_hi or stream_lo
    cudaStream_t stream_hi = nullptr, stream_lo = nullptr;
    cudaEvent_t ev_built = nullptr, ev_done = nullptr, ev_prep = nullptr;
    bool packable = false;           // its bin pass can join the round's packed launch
    int64_t* h_m = nullptr;         // pinned: edge count
    fsg_stats* h_stats = nullptr;   // pinned: statistics
    Pending p;
    Clock::time_point t_admit;
    bool cancel = false;
    fsg_tree* tree = nullptr;
    float* d_points = nullptr;
    int32_t* d_src = nullptr;
    int32_t* d_dst = nullptr;
    float* d_w = nullptr;
    int64_t* d_m = nullptr;
    fsg_stats* d_stats = nullptr;
};

size_t request_bytes(const fsg_request& r) {
    size_t b = fsg::tree_bytes_estimate(r.n, r.d, r.L) + sizeof(float) * (size_t)r.n * r.d +
               (sizeof(int32_t) * 2 + sizeof(float)) * (size_t)r.n * r.L + 4096;
    if (r.params.precision == FSG_PREC_SPLIT_BF16 && r.d <= 64)  // bins hold at least 32 points; the order's scratch
        b += fsg::split_workspace_bytes(r.n, (r.n + 31) / 32, r.d > 16) + fsg::spatial_order_scratch_bytes(r.n, r.d);
    else if (r.params.precision == FSG_PREC_SPLIT_BF16)  // d > 64: the three-part BF16 image and its norms
        b += (sizeof(uint16_t) * 3 * (size_t)((r.d + 63) / 64 * 64) + sizeof(float)) * (size_t)(r.n + 256);
    return b;
}

// Run-time estimate of one request alone: the bin pass and leaf work scale
// with n^2 (d + 6) pair operations (about 4.5e-11 ms each on one GB300 for the
// fused schedule), plus a fixed cost for the launches and copies.  Only the
// ratio between requests and against waiting time matters.
double request_est_ms(const fsg_request& r) {
    const double n = (double)r.n;
    return 0.25 + 4.5e-11 * n * n * (double)(r.d + 6);
}

}  // namespace

// Requests whose estimated run time alone is below this go to their slot's
// high-priority stream: the GPU's block scheduler then starts their CTAs
// ahead of pending CTAs of long requests, so short requests are not queued
// behind the long ones' launches.
constexpr double kShortRequestMs = 5.0;

struct fsg_server {
    fsg_server_opts opts{};
    int device = 0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t merge_stream = nullptr;  // the rounds' packed bin passes
    cudaEvent_t ev_merged = nullptr;
    int64_t merged_launches = 0, merged_requests = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> pending;
    std::deque<fsg_result> done;
    std::vector<uint64_t> cancel_ids;
    uint64_t next_id = 1;
    int64_t bytes_in_use = 0;
    int64_t admissions = 0;
    bool stop = false;
    std::thread worker;

    void finish(const Pending& p, int status, int64_t m, int64_t flagged, Clock::time_point t_admit) {
        fsg_result r{};
        r.id = p.id;
        r.status = status;
        r.n_edges = m;
        r.n_flagged = flagged;
        const auto now = Clock::now();
        r.latency_ms = ms_since(p.t_submit, now);
        r.queue_ms = ms_since(p.t_submit, t_admit);
        std::lock_guard<std::mutex> lock(mu);
        done.push_back(r);
        cv_done.notify_all();
    }

    void release(Slot& s) {
        if (s.tree) fsg_free_tree(s.tree);
        s.tree = nullptr;
        for (void* ptr : {(void*)s.d_points, (void*)s.d_src, (void*)s.d_dst, (void*)s.d_w, (void*)s.d_m,
                          (void*)s.d_stats})
            if (ptr) cudaFreeAsync(ptr, s.stream);
        s.d_points = nullptr;
        s.d_src = s.d_dst = nullptr;
        s.d_w = nullptr;
        s.d_m = nullptr;
        s.d_stats = nullptr;
        std::lock_guard<std::mutex> lock(mu);
        bytes_in_use -= (int64_t)s.p.bytes;
        s.state = 0;
    }

    // First part of an admission, on the slot's stream: device buffers,
    // points uploaded, tree built; for a request that takes the symmetric FP32
    // bin pass also its workspace, so the round can pack its bin pass.
    int admit_prepare(Slot& s) {
        const fsg_request& r = s.p.req;
        s.stream = s.p.est_ms < kShortRequestMs ? s.stream_hi : s.stream_lo;
        s.packable = false;
        ++admissions;
        if (opts.inject_alloc_fail_every > 0 && admissions % opts.inject_alloc_fail_every == 0) return FSG_ERR_OOM;
        const size_t cap = (size_t)r.n * r.L;
        cudaError_t e = cudaMallocFromPoolAsync((void**)&s.d_points, sizeof(float) * (size_t)r.n * r.d, pool, s.stream);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&s.d_src, sizeof(int32_t) * cap, pool, s.stream);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&s.d_dst, sizeof(int32_t) * cap, pool, s.stream);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&s.d_w, sizeof(float) * cap, pool, s.stream);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&s.d_m, sizeof(int64_t), pool, s.stream);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&s.d_stats, sizeof(fsg_stats), pool, s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.d_points, r.h_points, sizeof(float) * (size_t)r.n * r.d, cudaMemcpyHostToDevice,
                                s.stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? FSG_ERR_OOM : FSG_ERR_CUDA;
        }
        // split-precision requests up to d = 64 get the spatial tree order
        // (compact tiles for its centring; the form above d = 64 centres nothing)
        fsg_tree_opts topts{};
        topts.order = r.params.precision == FSG_PREC_SPLIT_BF16 && r.d <= 64 ? FSG_ORDER_SPATIAL
                                                                             : FSG_ORDER_IDENTITY;
        int rc = fsg::build_tree_internal(s.d_points, r.n, r.d, &topts, s.stream, pool, &s.tree);
        if (rc != FSG_OK) return rc;
        const fsg_params& p = r.params;
        if (r.d <= fsg::kMaxFmaDim && p.schedule == FSG_SCHED_FUSED && p.kde_eps == 0.f &&
            (p.precision == FSG_PREC_AUTO || p.precision == FSG_PREC_FP32) &&
            fsg::check_graph_call(s.tree, &p) == FSG_OK && fsg::kde_bins_sym_supported(s.tree)) {
            rc = fsg::ensure_workspace(s.tree, r.L, s.stream);
            if (rc != FSG_OK) return rc;
            if (cudaEventRecord(s.ev_prep, s.stream) != cudaSuccess) return FSG_ERR_CUDA;
            s.packable = true;
        }
        return FSG_OK;
    }

    // Second part: the graph build (its bin pass already done when the round
    // packed it), then the edge count and statistics to the host.
    int admit_finish(Slot& s, bool bins_done) {
        const fsg_request& r = s.p.req;
        const size_t cap = (size_t)r.n * r.L;
        int rc = fsg::build_graph_internal(s.tree, &r.params, r.L, r.seed, r.edge_mode, s.d_src, s.d_dst, s.d_w,
                                           (int64_t)cap, s.d_m, nullptr, nullptr, nullptr, s.d_stats, s.stream,
                                           bins_done);
        if (rc != FSG_OK) return rc;
        cudaError_t e = cudaMemcpyAsync(s.h_m, s.d_m, sizeof(int64_t), cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_stats, s.d_stats, sizeof(fsg_stats), cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(s.ev_built, s.stream);
        return e == cudaSuccess ? FSG_OK : FSG_ERR_CUDA;
    }

    void fail(Slot& s, int rc) {
        // the slot's stream may hold partial work: let it drain before reuse
        cudaStreamSynchronize(s.stream);
        cudaGetLastError();
        finish(s.p, rc, 0, 0, s.t_admit);
        release(s);
    }

    // Launches a round of admitted requests.  The requests that take the
    // symmetric FP32 bin pass are grouped by (d, kernel family); a group of
    // two or more gets one packed bin-pass launch over all its members' block
    // pairs (the members' streams join into the merge stream and fork again),
    // so requests that arrive together share the GPU in one launch instead of
    // each leaving it partly idle at its own launch's tail.
    void launch_round(std::vector<Slot*>& round) {
        for (Slot* s : round) {
            const int rc = admit_prepare(*s);
            if (rc != FSG_OK) {
                fail(*s, rc);
                s->packable = false;
                s->state = 0;
            }
        }
        std::vector<bool> done(round.size(), false);
        for (size_t i = 0; i < round.size(); ++i) {
            Slot* a = round[i];
            if (done[i] || a->state != 1 || !a->packable) continue;
            std::vector<size_t> grp;
            for (size_t j = i; j < round.size() && grp.size() < (size_t)fsg::kSymPackMax; ++j) {
                Slot* b = round[j];
                if (!done[j] && b->state == 1 && b->packable && b->p.req.d == a->p.req.d &&
                    b->p.req.params.kernel == a->p.req.params.kernel)
                    grp.push_back(j);
            }
            if (grp.size() < 2) continue;
            fsg::SymPackTable tab{};
            int total = 0;
            cudaError_t e = cudaSuccess;
            for (size_t g = 0; g < grp.size(); ++g) {
                Slot* m = round[grp[g]];
                const fsg_request& r = m->p.req;
                total += fsg::sym_pack_fill(m->tree, fsg::kernel_params_of(&r.params, r.L, r.seed), total, &tab.d[g]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(merge_stream, m->ev_prep, 0);
            }
            tab.count = (int)grp.size();
            if (e == cudaSuccess)
                e = fsg::launch_kde_bins_sym_packed(tab, total, a->p.req.d, a->p.req.params.kernel, merge_stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev_merged, merge_stream);
            for (size_t g = 0; g < grp.size() && e == cudaSuccess; ++g)
                e = cudaStreamWaitEvent(round[grp[g]]->stream, ev_merged, 0);
            if (e != cudaSuccess) {  // not packed after all: the members run their own bin passes
                cudaGetLastError();
                continue;
            }
            ++merged_launches;
            merged_requests += (int64_t)grp.size();
            for (size_t g : grp) {
                done[g] = true;
                const int rc = admit_finish(*round[g], true);
                if (rc != FSG_OK) fail(*round[g], rc);
            }
        }
        for (size_t i = 0; i < round.size(); ++i) {
            if (done[i] || round[i]->state != 1) continue;
            const int rc = admit_finish(*round[i], false);
            if (rc != FSG_OK) fail(*round[i], rc);
        }
    }

    bool cancelled(uint64_t id) {
        for (uint64_t c : cancel_ids)
            if (c == id) return true;
        return false;
    }

    void run() {
        cudaSetDevice(device);
        for (;;) {
            bool progress = false;
            for (Slot& s : slots) {
                if (s.state == 1) {
                    const cudaError_t q = cudaEventQuery(s.ev_built);
                    if (q == cudaErrorNotReady) continue;
                    progress = true;
                    if (q != cudaSuccess) {
                        cudaGetLastError();
                        finish(s.p, FSG_ERR_CUDA, 0, 0, s.t_admit);
                        release(s);
                        continue;
                    }
                    const int64_t m = *s.h_m;
                    const fsg_request& r = s.p.req;
                    if (m > r.cap) {
                        finish(s.p, FSG_ERR_CAPACITY, m, s.h_stats->n_flagged, s.t_admit);
                        release(s);
                        continue;
                    }
                    cudaError_t e = cudaSuccess;
                    if (m > 0) {
                        e = cudaMemcpyAsync(r.h_src, s.d_src, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s.stream);
                        if (e == cudaSuccess)
                            e = cudaMemcpyAsync(r.h_dst, s.d_dst, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s.stream);
                        if (e == cudaSuccess)
                            e = cudaMemcpyAsync(r.h_w, s.d_w, sizeof(float) * m, cudaMemcpyDeviceToHost, s.stream);
                    }
                    if (e == cudaSuccess) e = cudaEventRecord(s.ev_done, s.stream);
                    if (e != cudaSuccess) {
                        cudaGetLastError();
                        finish(s.p, FSG_ERR_CUDA, 0, 0, s.t_admit);
                        release(s);
                        continue;
                    }
                    s.state = 2;
                } else if (s.state == 2) {
                    const cudaError_t q = cudaEventQuery(s.ev_done);
                    if (q == cudaErrorNotReady) continue;
                    progress = true;
                    int status = q == cudaSuccess ? (int)s.h_stats->status : FSG_ERR_CUDA;
                    if (q != cudaSuccess) cudaGetLastError();
                    bool canc;
                    {
                        std::lock_guard<std::mutex> lock(mu);
                        canc = cancelled(s.p.id);
                    }
                    if (canc && status == FSG_OK) status = FSG_ERR_CANCELLED;
                    finish(s.p, status, *s.h_m, s.h_stats->n_flagged, s.t_admit);
                    release(s);
                }
            }
            // Admission: the next requests in the chosen order, slot and budget
            // permitting, launched together as one round.
            std::vector<Slot*> round;
            for (;;) {
                Slot* free_slot = nullptr;
                for (Slot& s : slots)
                    if (s.state == 0) { free_slot = &s; break; }
                Pending p;
                {
                    std::unique_lock<std::mutex> lock(mu);
                    if (!free_slot || pending.empty()) break;
                    size_t pick = 0;
                    if (opts.admission == FSG_ADMIT_RESPONSE_RATIO) {
                        const Clock::time_point now = Clock::now();
                        double best = -1.0;
                        for (size_t k = 0; k < pending.size(); ++k) {
                            const Pending& q = pending[k];
                            const double ratio = (ms_since(q.t_submit, now) + q.est_ms) / q.est_ms;
                            if (ratio > best) { best = ratio; pick = k; }  // ties keep arrival order
                        }
                    }
                    if (bytes_in_use + (int64_t)pending[pick].bytes > opts.hbm_budget_bytes) break;
                    p = pending[pick];
                    pending.erase(pending.begin() + (ptrdiff_t)pick);
                    bytes_in_use += (int64_t)p.bytes;
                }
                progress = true;
                Slot& s = *free_slot;
                s.p = p;
                s.t_admit = Clock::now();
                s.state = 1;
                s.stream = s.p.est_ms < kShortRequestMs ? s.stream_hi : s.stream_lo;
                round.push_back(&s);
            }
            if (!round.empty()) launch_round(round);
            {
                std::unique_lock<std::mutex> lock(mu);
                bool busy = false;
                for (Slot& s : slots) busy |= s.state != 0;
                if (stop && !busy) break;
                if (!progress) {
                    if (busy) cv_work.wait_for(lock, std::chrono::microseconds(50));
                    else cv_work.wait_for(lock, std::chrono::milliseconds(5));
                }
            }
        }
    }
};

extern "C" {

int fsg_server_create(const fsg_server_opts* opts, fsg_server** out) {
    if (!out || !opts || opts->hbm_budget_bytes <= 0 || opts->max_slots < 1 || opts->max_slots > 64 ||
        opts->queue_cap < 0 || opts->inject_alloc_fail_every < 0 ||
        (opts->admission != FSG_ADMIT_ARRIVAL && opts->admission != FSG_ADMIT_RESPONSE_RATIO))
        return FSG_ERR_INVALID_ARG;
    *out = nullptr;
    fsg_server* sv = new (std::nothrow) fsg_server();
    if (!sv) return FSG_ERR_OOM;
    sv->opts = *opts;
    if (sv->opts.queue_cap == 0) sv->opts.queue_cap = 65536;
    cudaGetDevice(&sv->device);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = sv->device;
    cudaError_t e = cudaMemPoolCreate(&sv->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = (uint64_t)opts->hbm_budget_bytes;  // memory stays cached in the pool up to the budget
        e = cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    int prio_low = 0, prio_high = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sv->merge_stream, cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->ev_merged, cudaEventDisableTiming);
    sv->slots.resize(opts->max_slots);
    for (Slot& s : sv->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s.stream_hi, cudaStreamNonBlocking, prio_high);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s.stream_lo, cudaStreamNonBlocking, prio_low);
        s.stream = s.stream_lo;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_built, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_prep, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&s.h_m, sizeof(int64_t), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&s.h_stats, sizeof(fsg_stats), cudaHostAllocDefault);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        fsg_server_destroy(sv);
        return e == cudaErrorMemoryAllocation ? FSG_ERR_OOM : FSG_ERR_CUDA;
    }
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return FSG_OK;
}

int fsg_server_submit(fsg_server* sv, const fsg_request* r, uint64_t* id_out) {
    if (!sv || !r || !id_out) return FSG_ERR_INVALID_ARG;
    if (!r->h_points || r->n < 1 || r->d < 1 || r->d > 4096 || r->L < 1 || r->L > 64 || !r->h_src || !r->h_dst ||
        !r->h_w)
        return FSG_ERR_INVALID_ARG;
    if (r->edge_mode != FSG_EDGES_SET && r->edge_mode != FSG_EDGES_MULTI) return FSG_ERR_INVALID_ARG;
    const fsg_params& p = r->params;
    if (!(p.sigma > 0.0) || p.sigma != p.sigma || p.sigma > 1e300) return FSG_ERR_INVALID_ARG;
    if (p.weight_f64) return FSG_ERR_INVALID_ARG;  // h_w is float32
    if (r->cap < r->n * (int64_t)r->L) return FSG_ERR_CAPACITY;
    Pending pd;
    pd.req = *r;
    pd.t_submit = Clock::now();
    pd.bytes = request_bytes(*r);
    pd.est_ms = request_est_ms(*r);
    if ((int64_t)pd.bytes > sv->opts.hbm_budget_bytes) return FSG_ERR_BUSY;  // could never be admitted
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if ((int64_t)sv->pending.size() >= sv->opts.queue_cap) return FSG_ERR_BUSY;
        pd.id = sv->next_id++;
        sv->pending.push_back(pd);
    }
    sv->cv_work.notify_one();
    *id_out = pd.id;
    return FSG_OK;
}

int fsg_server_poll(fsg_server* sv, fsg_result* out, int32_t max, int32_t* count_out, int32_t wait_ms) {
    if (!sv || !count_out || max < 0 || (max > 0 && !out)) return FSG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(sv->mu);
    if (sv->done.empty() && wait_ms > 0)
        sv->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [sv] { return !sv->done.empty(); });
    int32_t k = 0;
    while (k < max && !sv->done.empty()) {
        out[k++] = sv->done.front();
        sv->done.pop_front();
    }
    *count_out = k;
    return FSG_OK;
}

int fsg_server_cancel(fsg_server* sv, uint64_t id) {
    if (!sv) return FSG_ERR_INVALID_ARG;
    Pending dropped;
    bool found = false;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it) {
            if (it->id == id) {
                dropped = *it;
                sv->pending.erase(it);
                found = true;
                break;
            }
        }
        if (!found) sv->cancel_ids.push_back(id);
    }
    if (found) sv->finish(dropped, FSG_ERR_CANCELLED, 0, 0, Clock::now());
    return FSG_OK;
}

int fsg_server_info(fsg_server* sv, int64_t* pending, int64_t* in_flight, int64_t* bytes_in_use) {
    if (!sv) return FSG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    if (pending) *pending = (int64_t)sv->pending.size();
    if (in_flight) {
        int64_t c = 0;
        for (const Slot& s : sv->slots) c += s.state != 0;
        *in_flight = c;
    }
    if (bytes_in_use) *bytes_in_use = sv->bytes_in_use;
    return FSG_OK;
}

void fsg_server_destroy(fsg_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->pending.clear();
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    if (sv->merge_stream) cudaStreamSynchronize(sv->merge_stream);
    for (Slot& s : sv->slots) {
        for (cudaStream_t st : {s.stream_hi, s.stream_lo}) {
            if (st) cudaStreamSynchronize(st);
            if (st) cudaStreamDestroy(st);
        }
        if (s.ev_built) cudaEventDestroy(s.ev_built);
        if (s.ev_done) cudaEventDestroy(s.ev_done);
        if (s.ev_prep) cudaEventDestroy(s.ev_prep);
        if (s.h_m) cudaFreeHost(s.h_m);
        if (s.h_stats) cudaFreeHost(s.h_stats);
    }
    if (sv->merge_stream) cudaStreamDestroy(sv->merge_stream);
    if (sv->ev_merged) cudaEventDestroy(sv->ev_merged);
    if (sv->pool) cudaMemPoolDestroy(sv->pool);
    delete sv;
}

}  // extern "C"
