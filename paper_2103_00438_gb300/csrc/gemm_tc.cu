// libwfq entry to the tcgen05 GEMMs of gemm_tc.cuh and gemm_mf.cuh (the dense product of
// the mixed operator, U = D X with three bf16 products), with their autotuner: the first
// product of a shape on a context times the pipeline depths below on the real operands and
// keeps the fastest for later products of that shape.  The depth changes only how far the
// loads run ahead of the tensor cores, never which products are summed in which order, so
// the choice cannot change a result.
#include <vector>

#include "common.h"
#include "gemm_mf.cuh"
#include "gemm_tc.cuh"

namespace wfq {

namespace {

// pipeline depths tried (0: as deep as shared memory allows, at most the kernels' maximum)
constexpr int kStageChoices[] = {0, 4, 3, 2};

template <class Launch>
int tuned_stages(const wfq_geom *g, int64_t key, cudaStream_t s, Launch launch) {
    {
        std::lock_guard<std::mutex> lk(g->ctx->tune_mu);
        auto it = g->ctx->tuned.find(key);
        if (it != g->ctx->tuned.end()) return it->second;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return 0;
    }
    int best = 0;
    float best_ms = 1e30f;
    for (int st : kStageChoices) {
        float ms = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {   // the first of the three warms up
            if (rep == 1) cudaEventRecord(e0, s);
            ok = launch(st) == cudaSuccess;
        }
        cudaEventRecord(e1, s);
        if (!ok || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = st;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g->ctx->tune_mu);
    g->ctx->tuned[key] = best;
    return best;
}

// autotuner keys of the GEMMs: bit 60 set (the GEMV keys stay below 2^40), kernel id, shape
inline int64_t gemm_key(int kernel, int64_t npad, int64_t cpad) {
    return ((int64_t)1 << 60) | ((int64_t)kernel << 56) | (npad << 20) | cpad;
}

}  // namespace

int gemm_3xbf16_mf(const wfq_geom *g, int64_t cpad, const __nv_bfloat16 *Xhi, const __nv_bfloat16 *Xlo, float *U,
                   int64_t ldu, cudaStream_t s) {
    std::string msg;
    int launches = 0;
    // timing twelve launches costs seconds at a million atoms (1.4 s per launch): large
    // shapes take the deepest pipeline without a trial
    const int st = g->npad > 262144 ? 0 : tuned_stages(g, gemm_key(2, g->npad, cpad), s, [&](int stg) {
        int l = 0;
        const cudaError_t e = tc::gemm3_mf(g->atom32, g->atom32p, g->n, g->npad, Xhi, Xlo, cpad, U, ldu, g->ctx->num_sms,
                                           g->ctx->dev_err, s, &l, nullptr, stg);
        for (int i = 0; i < l; ++i) note_launch();
        return e;
    });
    KScope ks(g->ctx, WFQ_KT_GEMM_MIXED, s, 6.0 * (double)g->n * (double)g->n * (double)ldu);
    cudaError_t e = tc::gemm3_mf(g->atom32, g->atom32p, g->n, g->npad, Xhi, Xlo, cpad, U, ldu, g->ctx->num_sms, g->ctx->dev_err,
                                 s, &launches, &msg, st);
    for (int i = 0; i < launches; ++i) note_launch();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(WFQ_ECUDA, "matrix-free tensor-core GEMM: " + (msg.empty() ? std::string(cudaGetErrorString(e)) : msg));
    }
    return WFQ_OK;
}

int gemm_3xbf16(const wfq_geom *g, int64_t cpad, const __nv_bfloat16 *Xhi, const __nv_bfloat16 *Xlo, float *U,
                int64_t ldu, cudaStream_t s) {
    std::string msg;
    int launches = 0;
    const int st = tuned_stages(g, gemm_key(1, g->npad, cpad), s, [&](int stg) {
        int l = 0;
        const cudaError_t e = tc::gemm3_tc(g->Dhi, g->Dlo, g->n, g->npad, Xhi, Xlo, cpad, U, ldu, g->ctx->num_sms,
                                           g->ctx->dev_err, s, &l, nullptr, stg);
        for (int i = 0; i < l; ++i) note_launch();
        return e;
    });
    KScope ks(g->ctx, WFQ_KT_GEMM_MIXED, s, 6.0 * (double)g->n * (double)g->n * (double)ldu);
    cudaError_t e = tc::gemm3_tc(g->Dhi, g->Dlo, g->n, g->npad, Xhi, Xlo, cpad, U, ldu, g->ctx->num_sms,
                                 g->ctx->dev_err, s, &launches, &msg, st);
    for (int i = 0; i < launches; ++i) note_launch();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(WFQ_ECUDA, "tensor-core GEMM: " + (msg.empty() ? std::string(cudaGetErrorString(e)) : msg));
    }
    return WFQ_OK;
}

}  // namespace wfq
