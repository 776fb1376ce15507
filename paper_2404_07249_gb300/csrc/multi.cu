// Batched ideal bispectra over fields on (possibly) different grids: the whole batch -- per field the pruned
// forward transform, the shell maps, the triplet contraction and the copy of its result to pinned host memory --
// is captured once into a CUDA graph on a private stream and replayed there with a single graph launch, ordered
// after the work already queued on the contexts' stream.
// The graph is cached in the first context, keyed by the context ids and field pointers of the call.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstring>
#include <vector>

#include "polybin_internal.h"

namespace pb {

struct MultiCache {
    std::vector<unsigned long long> key;
    cudaStream_t cap = nullptr;             // private stream: capture and replay (the legacy stream cannot capture)
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t exec = nullptr;
    double* host = nullptr;                 // pinned: contraction results of every field
    std::vector<size_t> off;                // per-field offset into host
};

void destroy_multi(polybin_ctx* ctx) {
    MultiCache* m = static_cast<MultiCache*>(ctx->multi);
    if (!m) return;
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->host) cudaFreeHost(m->host);
    if (m->ev) cudaEventDestroy(m->ev);
    if (m->cap) cudaStreamDestroy(m->cap);
    delete m;
    ctx->multi = nullptr;
}

template <typename T>
static int capture_field(polybin_ctx* c, const float* field, double* host_dst) {
    int rc;
    Work& w = c->w;
    const size_t nt = c->Nabc.size();
    if (nt == 0) return POLYBIN_OK;
    if ((rc = run_forward<T, float, float>(c, field, (const float*)nullptr, (const float*)nullptr, (C<T>*)w.t1, (C<T>*)w.t2,
                                           (C<T>*)w.box)))
        return rc;
    if ((rc = run_shells<T>(c, (const C<T>*)w.box, (C<T>*)w.u1, (C<T>*)w.u2, (T*)w.g, 0, c->cg))) return rc;
    if ((rc = run_triplet_sums<T>(c, (const T*)w.g, c->d_S))) return rc;
    if ((rc = run_bk_normalise(c, c->d_S, c->d_B))) return rc;
    cudaError_t e = cudaMemcpyAsync(host_dst, c->d_B, sizeof(double) * nt, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "capture copy", __FILE__, __LINE__);
    return POLYBIN_OK;
}

}  // namespace pb

using namespace pb;

extern "C" int polybin_bk_ideal_multi(polybin_ctx* const* ctxs, const float* const* fields, int n_fields,
                                      double* const* bk_out) {
    if (!ctxs || !fields || !bk_out || n_fields < 1 || !ctxs[0])
        return fail(nullptr, POLYBIN_EINVAL, "polybin_bk_ideal_multi: bad argument");
    polybin_ctx* c0 = ctxs[0];
    int rc;
    std::vector<unsigned long long> key;
    key.reserve(2 * (size_t)n_fields + 1);
    key.push_back((unsigned long long)n_fields);
    for (int i = 0; i < n_fields; ++i) {
        polybin_ctx* c = ctxs[i];
        if (!c || !fields[i] || !bk_out[i]) return fail(c0, POLYBIN_EINVAL, "polybin_bk_ideal_multi: NULL entry %d", i);
        if (c->stream != c0->stream) return fail(c0, POLYBIN_EINVAL, "polybin_bk_ideal_multi: contexts must share one stream");
        if (c->profiling) return fail(c0, POLYBIN_EINVAL, "polybin_bk_ideal_multi: disable profiling first");
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, fields[i]) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(c0, POLYBIN_EINVAL, "polybin_bk_ideal_multi: field %d must be device memory", i);
        }
        if ((rc = ensure_triplets(c))) return rc;
        if ((rc = ensure_err_flag(c))) return rc;
        key.push_back(c->uid);
        key.push_back((unsigned long long)(uintptr_t)fields[i]);
    }
    MultiCache* m = static_cast<MultiCache*>(c0->multi);
    if (!m || m->key != key) {
        destroy_multi(c0);
        m = new (std::nothrow) MultiCache();
        if (!m) return fail(c0, POLYBIN_ENOMEM, "polybin_bk_ideal_multi: out of host memory");
        c0->multi = m;
        m->key = key;
        size_t total = 0;
        for (int i = 0; i < n_fields; ++i) {
            m->off.push_back(total);
            total += std::max(ctxs[i]->Nabc.size(), (size_t)1);
        }
        {
            polybin_ctx* ctx = c0;
            PB_CUDA_OK(cudaHostAlloc((void**)&m->host, sizeof(double) * total, cudaHostAllocDefault));
        }
        {
            polybin_ctx* ctx = c0;
            PB_CUDA_OK(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
            PB_CUDA_OK(cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming));
        }
        cudaStream_t st = m->cap;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGetLastError();
            destroy_multi(c0);
            return fail_cuda(c0, e, "cudaStreamBeginCapture", __FILE__, __LINE__);
        }
        std::vector<cudaStream_t> saved(n_fields);
        for (int i = 0; i < n_fields; ++i) { saved[i] = ctxs[i]->stream; ctxs[i]->stream = st; ctxs[i]->capturing = true; }
        rc = POLYBIN_OK;
        for (int i = 0; i < n_fields && !rc; ++i) {
            polybin_ctx* c = ctxs[i];
            rc = c->prec == POLYBIN_FP64 ? capture_field<double>(c, fields[i], m->host + m->off[i])
                                         : capture_field<float>(c, fields[i], m->host + m->off[i]);
            if (rc && c != c0) c0->err = c->err;
        }
        for (int i = 0; i < n_fields; ++i) { ctxs[i]->capturing = false; ctxs[i]->stream = saved[i]; }
        e = cudaStreamEndCapture(st, &graph);
        if (rc || e != cudaSuccess) cudaGetLastError();
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            destroy_multi(c0);
            return rc;
        }
        if (e != cudaSuccess) { destroy_multi(c0); return fail_cuda(c0, e, "cudaStreamEndCapture", __FILE__, __LINE__); }
        e = cudaGraphInstantiate(&m->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { destroy_multi(c0); return fail_cuda(c0, e, "cudaGraphInstantiate", __FILE__, __LINE__); }
    }
    // fence: the graph starts after the work already queued on the caller's stream
    cudaError_t e = cudaEventRecord(m->ev, c0->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->cap, m->ev, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(m->exec, m->cap);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->cap);
    if (e != cudaSuccess) return fail_cuda(c0, e, "cudaGraphLaunch", __FILE__, __LINE__);
    for (int i = 0; i < n_fields; ++i) {
        polybin_ctx* c = ctxs[i];
        int herr[kErrFlags] = {0, 0};
        {
            polybin_ctx* ctx = c0;
            PB_CUDA_OK(cudaMemcpy(herr, c->d_err, sizeof(herr), cudaMemcpyDeviceToHost));
            if (herr[kErrStaging]) PB_CUDA_OK(cudaMemset(c->d_err + kErrStaging, 0, sizeof(int)));
        }
        if (herr[kErrPipeline] || herr[kErrStaging])
            return fail(c0, POLYBIN_ETIMEOUT, "polybin_bk_ideal_multi: a %s wait timed out (field %d)",
                        herr[kErrStaging] ? "bulk staging" : "pipeline", i);
        const double* B = m->host + m->off[i];
        std::memcpy(bk_out[i], B, sizeof(double) * c->Nabc.size());
    }
    return POLYBIN_OK;
}
