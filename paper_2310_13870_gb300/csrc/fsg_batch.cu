// Batched graph construction (fsg_batch_*): one tree per point set, the sets'
// launch sequences spread over several streams forked from the caller's
// stream, and optionally captured once into a CUDA graph and replayed.
#include <new>
#include <vector>

#include "fsg_internal.cuh"

struct fsg_batch {
    std::vector<fsg_batch_item> items;
    std::vector<fsg_tree*> trees;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;   // one per internal stream (join)
    cudaEvent_t fork = nullptr;
    int capture = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool warmed = false;
    // Packed bin pass: when every set takes the symmetric FP32 pass (same d
    // and kernel family), one launch computes all sets' bin sums, its CTAs
    // taking the block pairs of every set's triangle in turn, so no set's
    // launch leaves the GPU partly idle at its tail.
    fsg::SymPackDesc* d_descs = nullptr;
    int pack_total = 0;              // block pairs over all sets (0: not packed)
    int pack_d = 0, pack_family = 0;
};

namespace {

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return FSG_OK;
    if (e == cudaErrorMemoryAllocation) return FSG_ERR_OOM;
    return FSG_ERR_CUDA;
}

cudaError_t fork_streams(fsg_batch* b, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (size_t k = 0; e == cudaSuccess && k < b->streams.size(); ++k) e = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
    return e;
}

cudaError_t join_streams(fsg_batch* b, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; e == cudaSuccess && k < b->streams.size(); ++k) {
        e = cudaEventRecord(b->done[k], b->streams[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->done[k], 0);
    }
    return e;
}

// Enqueues every set on the internal streams, forked from / joined into s.
// Packed: the trees' refresh on the streams, the one bin-pass launch on s,
// then the rest of every set's graph build on the streams again.
int enqueue_all(fsg_batch* b, cudaStream_t s) {
    cudaError_t e = fork_streams(b, s);
    if (e != cudaSuccess) return status_of(e);
    const bool packed = b->pack_total > 0;
    for (size_t i = 0; i < b->items.size(); ++i) {
        const fsg_batch_item& it = b->items[i];
        cudaStream_t si = b->streams[i % b->streams.size()];
        int rc = fsg_tree_update(b->trees[i], it.d_points, si);
        if (rc == FSG_OK && !packed)
            rc = fsg_build_graph(b->trees[i], &it.params, it.L, it.seed, it.edge_mode, it.d_src, it.d_dst, it.d_w,
                                 it.cap, it.d_m_out, it.d_deg, nullptr, nullptr, it.d_stats, si);
        if (rc != FSG_OK) return rc;
    }
    if (packed) {
        e = join_streams(b, s);
        if (e == cudaSuccess)
            e = fsg::launch_kde_bins_sym_packed(b->d_descs, (int)b->items.size(), b->pack_total, b->pack_d,
                                                b->pack_family, s);
        if (e == cudaSuccess) e = fork_streams(b, s);
        if (e != cudaSuccess) return status_of(e);
        for (size_t i = 0; i < b->items.size(); ++i) {
            const fsg_batch_item& it = b->items[i];
            cudaStream_t si = b->streams[i % b->streams.size()];
            const int rc = fsg::build_graph_internal(b->trees[i], &it.params, it.L, it.seed, it.edge_mode, it.d_src,
                                                     it.d_dst, it.d_w, it.cap, it.d_m_out, it.d_deg, nullptr,
                                                     nullptr, it.d_stats, si, true);
            if (rc != FSG_OK) return rc;
        }
    }
    e = join_streams(b, s);
    return e == cudaSuccess ? FSG_OK : status_of(e);
}

// Sets up the packed bin pass when every set qualifies (see fsg_batch).
int setup_pack(fsg_batch* b, cudaStream_t s) {
    const int d = b->items[0].d, fam = b->items[0].params.kernel;
    for (size_t i = 0; i < b->items.size(); ++i) {
        const fsg_batch_item& it = b->items[i];
        const fsg_params& p = it.params;
        if (it.d != d || it.d > fsg::kMaxFmaDim || p.kernel != fam || p.schedule != FSG_SCHED_FUSED ||
            (p.precision != FSG_PREC_AUTO && p.precision != FSG_PREC_FP32) || p.kde_eps != 0.f ||
            fsg::check_graph_call(b->trees[i], &p) != FSG_OK || !fsg::kde_bins_sym_supported(b->trees[i]))
            return FSG_OK;  // not packed: every set keeps its own launches
    }
    std::vector<fsg::SymPackDesc> descs(b->items.size());
    int total = 0;
    for (size_t i = 0; i < b->items.size(); ++i) {
        const fsg_batch_item& it = b->items[i];
        const int rc = fsg::ensure_workspace(b->trees[i], it.L, s);  // the bin sums' address is fixed from here on
        if (rc != FSG_OK) return rc;
        total += fsg::sym_pack_fill(b->trees[i], fsg::kernel_params_of(&it.params, it.L, it.seed), total, &descs[i]);
    }
    cudaError_t e = cudaMalloc((void**)&b->d_descs, sizeof(fsg::SymPackDesc) * descs.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_descs, descs.data(), sizeof(fsg::SymPackDesc) * descs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return status_of(e);
    }
    b->pack_total = total;
    b->pack_d = d;
    b->pack_family = fam;
    return FSG_OK;
}

}  // namespace

extern "C" {

void fsg_batch_destroy(fsg_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto* t : b->trees) fsg_free_tree(t);
    if (b->d_descs) cudaFree(b->d_descs);
    for (auto st : b->streams) cudaStreamDestroy(st);
    for (auto ev : b->done) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

int fsg_batch_create(const fsg_batch_item* items, int32_t count, int32_t streams, int32_t capture, void* stream,
                     fsg_batch** out) {
    if (!out) return FSG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!items || count < 1 || streams < 1 || streams > 64) return FSG_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i) {
        const fsg_batch_item& it = items[i];
        if (!it.d_points || it.n < 1 || it.d < 1 || it.L < 1 || it.L > 64 || !it.d_src || !it.d_dst || !it.d_w ||
            !it.d_m_out)
            return FSG_ERR_INVALID_ARG;
        if (it.edge_mode != FSG_EDGES_SET && it.edge_mode != FSG_EDGES_MULTI) return FSG_ERR_INVALID_ARG;
        if (it.params.weight_f64) return FSG_ERR_INVALID_ARG;  // d_w is float32
        if (it.cap < it.n * (int64_t)it.L) return FSG_ERR_CAPACITY;
    }
    fsg_batch* b = new (std::nothrow) fsg_batch();
    if (!b) return FSG_ERR_OOM;
    b->items.assign(items, items + count);
    b->capture = capture;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int32_t k = 0; e == cudaSuccess && k < streams && k < count; ++k) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->streams.push_back(st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->done.push_back(ev);
    }
    if (e != cudaSuccess) {
        fsg_batch_destroy(b);
        return status_of(e);
    }
    for (int32_t i = 0; i < count; ++i) {
        fsg_tree* t = nullptr;
        int rc = fsg_build_tree(items[i].d_points, items[i].n, items[i].d, nullptr, stream, &t);
        if (rc != FSG_OK) {
            fsg_batch_destroy(b);
            return rc;
        }
        b->trees.push_back(t);
    }
    const int rc = setup_pack(b, (cudaStream_t)stream);
    if (rc != FSG_OK) {
        fsg_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FSG_OK;
}

int fsg_batch_run(fsg_batch* b, void* stream) {
    if (!b) return FSG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->capture || !b->warmed) {
        // First run (or no capture): plain enqueue; workspaces grow here.
        const int rc = enqueue_all(b, s);
        b->warmed = true;
        return rc;
    }
    if (!b->exec) {
        // Capture on a private stream (the legacy default stream cannot be captured).
        cudaStream_t cs = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return status_of(e);
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? enqueue_all(b, cs) : status_of(e);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (rc != FSG_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e2 != cudaSuccess) return status_of(e2);
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return status_of(e);
        }
    }
    return status_of(cudaGraphLaunch(b->exec, s));
}

}  // extern "C"
