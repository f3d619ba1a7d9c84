// libwfq entry to the tcgen05 GEMM of gemm_tc.cuh (the dense product of the mixed
// operator, U = D X with three bf16 products).
#include "common.h"
#include "gemm_mf.cuh"
#include "gemm_tc.cuh"

namespace wfq {

int gemm_3xbf16_mf(const wfq_geom *g, int64_t cpad, const __nv_bfloat16 *Xhi, const __nv_bfloat16 *Xlo, float *U,
                   int64_t ldu, cudaStream_t s) {
    std::string msg;
    int launches = 0;
    KScope ks(g->ctx, WFQ_KT_GEMM_MIXED, s, 6.0 * (double)g->n * (double)g->n * (double)ldu);
    cudaError_t e = tc::gemm3_mf(g->atom32, g->n, g->npad, Xhi, Xlo, cpad, U, ldu, g->ctx->num_sms, g->ctx->dev_err,
                                 s, &launches, &msg);
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
    KScope ks(g->ctx, WFQ_KT_GEMM_MIXED, s, 6.0 * (double)g->n * (double)g->n * (double)ldu);
    cudaError_t e = tc::gemm3_tc(g->Dhi, g->Dlo, g->n, g->npad, Xhi, Xlo, cpad, U, ldu, g->ctx->num_sms,
                                 g->ctx->dev_err, s, &launches, &msg);
    for (int i = 0; i < launches; ++i) note_launch();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(WFQ_ECUDA, "tensor-core GEMM: " + (msg.empty() ? std::string(cudaGetErrorString(e)) : msg));
    }
    return WFQ_OK;
}

}  // namespace wfq
