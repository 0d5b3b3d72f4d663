// Per-kernel-class timing with CUDA events recorded on the context's stream.
#include "fs_common.cuh"

#include <cstring>

namespace {
const char* const KS_NAMES[KS_COUNT] = {"col_inverse_fft", "plane_fft_vloc", "col_forward_fft",
                                        "nonlocal_project", "nonlocal_D",    "nonlocal_add",
                                        "gram",            "rotate",         "vector",
                                        "dense_la",        "col_inverse_fft_fp64", "plane_fft_vloc_fp64",
                                        "col_forward_fft_fp64", "nonlocal_project_fp64", "nonlocal_add_fp64",
                                        "gram_fp64",       "rotate_fp64",    "vector_fp64",
                                        "dense.potrf",     "dense.trsm",     "dense.hetrd",
                                        "dense.tridiag_eig", "dense.backtransform"};

cudaEvent_t take(fs_ctx* c) {
    if (!c->prof.pool.empty()) {
        cudaEvent_t e = c->prof.pool.back();
        c->prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    FS_CUDA(cudaEventCreate(&e));
    return e;
}
}  // namespace

ProfScope::ProfScope(fs_ctx* c_, int id_, double bytes, double flops) : c(c_), id(id_) {
    if (!c || !c->prof.on) return;
    KStat& k = c->prof.st[id];
    k.launches += 1;
    k.bytes += bytes;
    k.flops += flops;
    a = take(c);
    cudaEventRecord(a, c->stream);
}

ProfScope::~ProfScope() {
    if (!a) return;
    cudaEvent_t b = nullptr;
    if (!c->prof.pool.empty()) {
        b = c->prof.pool.back();
        c->prof.pool.pop_back();
    } else if (cudaEventCreate(&b) != cudaSuccess) {
        c->prof.pool.push_back(a);
        return;
    }
    cudaEventRecord(b, c->stream);
    c->prof.pend.push_back({id, a, b});
    if (c->prof.pend.size() > 4096) prof_flush(c);
}

void prof_flush(fs_ctx* c) {
    if (c->prof.pend.empty()) return;
    FS_CUDA(cudaStreamSynchronize(c->stream));
    for (auto& p : c->prof.pend) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->prof.st[p.id].ms += ms;
        c->prof.pool.push_back(p.a);
        c->prof.pool.push_back(p.b);
    }
    c->prof.pend.clear();
}

void prof_release(fs_ctx* c) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& p : c->prof.pend) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    c->prof.pend.clear();
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    c->prof.pool.clear();
}

extern "C" {

fs_status fs_profile(fs_ctx* c, int enable) {
    if (!c) return FS_ERR_ARG;
    try {
        prof_flush(c);
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    }
    for (auto& k : c->prof.st) k = KStat();
    c->prof.on = enable != 0;
    return FS_OK;
}

fs_status fs_kernel_stats(fs_ctx* c, fs_kernel_stat* out, int max, int* count) {
    if (!c || !count || (max > 0 && !out) || max < 0) return FS_ERR_ARG;
    try {
        prof_flush(c);
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    }
    *count = KS_COUNT;
    for (int i = 0; i < KS_COUNT && i < max; ++i) {
        out[i].name = KS_NAMES[i];
        out[i].launches = c->prof.st[i].launches;
        out[i].ms = c->prof.st[i].ms;
        out[i].bytes = c->prof.st[i].bytes;
        out[i].flops = c->prof.st[i].flops;
    }
    return FS_OK;
}

}  // extern "C"
