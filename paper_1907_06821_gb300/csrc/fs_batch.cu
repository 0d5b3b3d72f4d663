// Batched independent boxes (the linear-scaling divide-and-conquer setting of
// the paper's LS3DF step, Sec. II.B, where many fragment problems of uneven
// size are solved independently): a batch groups contexts, each with its own
// stream, and solves them concurrently from a pool of host threads so that the
// GPU runs several boxes' kernels at once.  Also the FFT column-tile autotuner.
#include "fs_common.cuh"

#include <algorithm>
#include <cstdio>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

struct fs_batch {
    std::vector<fs_ctx*> ctx;
    int nthreads = 1;
    std::string err;
};

namespace {
std::mutex g_tune_mu;
struct Tuned {
    int cpb, ipt;
    size_t chunk;
};
std::map<std::tuple<int, int, int, int, int>, Tuned> g_tuned;  // (n0, n1, n2, ncol, fp32) -> launch shapes

template <typename T2> double time_apply(fs_ctx* c, int nb, int reps) {
    dbuf in, out;
    in.alloc((size_t)nb * c->npw * sizeof(T2));
    out.alloc((size_t)nb * c->npw * sizeof(T2));
    FS_CUDA(cudaMemsetAsync(in.p, 0, in.bytes, c->stream));
    apply_H_impl<T2>(c, in.as<T2>(), out.as<T2>(), nb, 0.0);  // warm
    cudaEvent_t a, b;
    FS_CUDA(cudaEventCreate(&a));
    FS_CUDA(cudaEventCreate(&b));
    FS_CUDA(cudaEventRecord(a, c->stream));
    for (int r = 0; r < reps; ++r) apply_H_impl<T2>(c, in.as<T2>(), out.as<T2>(), nb, 0.0);
    FS_CUDA(cudaEventRecord(b, c->stream));
    FS_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}
}  // namespace

extern "C" {

// Pick the FFT launch shapes for this context's grid by timing H applications
// of 32 bands with each candidate (coordinate descent: column tile of the z
// kernels, then line items per thread of the plane kernel, then the band
// chunk whose column buffer stays in L2); results are cached per grid shape
// and precision for the process.  verbose > 0 prints each timing on stderr.
fs_status fs_autotune(fs_ctx* c, int* cpb_out) {
    if (!c) return FS_ERR_ARG;
    try {
        const bool fp32 = c->opt.precision == FS_MIXED;
        auto key = std::make_tuple(c->n[0], c->n[1], c->n[2], c->ncol, (int)fp32);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                c->cpb = it->second.cpb;
                c->pf_ipt = it->second.ipt;
                c->hchunk_bytes = it->second.chunk;
                if (cpb_out) *cpb_out = c->cpb;
                return FS_OK;
            }
        }
        const int nb = 32;
        auto time_now = [&]() { return fp32 ? time_apply<float2>(c, nb, 3) : time_apply<double2>(c, nb, 3); };
        auto report = [&](const char* what, int v, double ms) {
            if (c->opt.verbose) fprintf(stderr, "[fs] autotune %s %d: %.3f ms for %d bands\n", what, v, ms, nb);
        };
        // column tile; it serves both precisions of a mixed solve, so it is sized for FP64
        int best = c->cpb;
        double best_ms = 1e300;
        for (int cand : {2, 4, 8, 16, 32}) {
            const size_t need = c->fast ? ((size_t)cand * c->Pz + c->n[2]) * sizeof(double2)
                                        : (size_t)cand * c->n[2] * sizeof(double2);
            if (need > 200 * 1024) continue;
            c->cpb = cand;
            const double ms = time_now();
            report("z-column tile", cand, ms);
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        c->cpb = best;
        if (c->fast) {
            int bi = c->pf_ipt;
            for (int ipt : {1, 2, 3, 4}) {
                c->pf_ipt = ipt;
                const double ms = time_now();
                report("plane items per thread", ipt, ms);
                if (ms < best_ms) {
                    best_ms = ms;
                    bi = ipt;
                }
            }
            c->pf_ipt = bi;
            size_t bc = c->hchunk_bytes;
            for (size_t mb : {16, 32, 48, 64, 96}) {
                c->hchunk_bytes = mb << 20;
                const double ms = time_now();
                report("chunk MiB", (int)mb, ms);
                if (ms < best_ms) {
                    best_ms = ms;
                    bc = mb << 20;
                }
            }
            c->hchunk_bytes = bc;
        }
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key] = Tuned{c->cpb, c->pf_ipt, c->hchunk_bytes};
        }
        if (cpb_out) *cpb_out = c->cpb;
        c->err.clear();
        return FS_OK;
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    }
}

fs_status fs_batch_create(int nbox, fs_ctx* const* ctxs, int nthreads, fs_batch** out) {
    if (!out) return FS_ERR_ARG;
    *out = nullptr;
    if (nbox <= 0 || !ctxs) return FS_ERR_ARG;
    for (int i = 0; i < nbox; ++i) {
        if (!ctxs[i]) return FS_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i] || ctxs[j]->stream == ctxs[i]->stream) return FS_ERR_ARG;
    }
    fs_batch* b = new (std::nothrow) fs_batch();
    if (!b) return FS_ERR_OOM;
    b->ctx.assign(ctxs, ctxs + nbox);
    b->nthreads = std::max(1, std::min(nthreads > 0 ? nthreads : 8, nbox));
    *out = b;
    return FS_OK;
}

// Solve every box concurrently: box i for e_ref[i], nstates[i]; res[i] must
// hold nstates[i] doubles in eps and resid; status[i] receives the box's
// status.  Returns FS_OK when every box converged, else the first non-OK status.
fs_status fs_batch_solve(fs_batch* b, const double* e_ref, const int* nstates, double tol, fs_result* res,
                         fs_status* status) {
    if (!b || !e_ref || !nstates || !res || !status || !(tol > 0)) return FS_ERR_ARG;
    const int n = (int)b->ctx.size();
    std::atomic<int> next(0);
    auto worker = [&]() {
        for (;;) {
            int i = next.fetch_add(1);
            if (i >= n) break;
            status[i] = fs_solve(b->ctx[i], e_ref[i], nstates[i], tol, &res[i]);
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < b->nthreads; ++t) th.emplace_back(worker);
    for (auto& t : th) t.join();
    fs_status first = FS_OK;
    for (int i = 0; i < n; ++i)
        if (status[i] != FS_OK && first == FS_OK) first = status[i];
    return first;
}

void fs_batch_destroy(fs_batch* b) { delete b; }

}  // extern "C"
