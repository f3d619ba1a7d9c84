// U = Dhi.Xhi + Dhi.Xlo + Dlo.Xhi with FP32 accumulation on the CUDA cores (64 x 64
// tiles).  The bf16 planes hold D ~= Dhi + Dlo and X ~= Xhi + Xlo (16 significant
// bits each); the dropped lo.lo product is below 2^-16 relative.
#include "common.h"

namespace wfq {

__global__ void __launch_bounds__(256) k_gemm3_simt(int64_t n, int64_t npad, int64_t ldu,
                                                    const __nv_bfloat16 *__restrict__ Dhi,
                                                    const __nv_bfloat16 *__restrict__ Dlo,
                                                    const __nv_bfloat16 *__restrict__ Xhi,
                                                    const __nv_bfloat16 *__restrict__ Xlo, float *__restrict__ U) {
    __shared__ float Ah[32][65], Al[32][65], Bh[32][64], Bl[32][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    float acc[4][4] = {};
    for (int64_t k0 = 0; k0 < npad; k0 += 32) {
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            int e = tid + l * 256;
            int r = e >> 5, kk = e & 31;
            int64_t ia = (m0 + r) * npad + k0 + kk;   // rows < npad by construction
            Ah[kk][r] = __bfloat162float(Dhi[ia]);
            Al[kk][r] = __bfloat162float(Dlo[ia]);
            int64_t ib = (c0 + r) * npad + k0 + kk;   // X planes have cpad rows
            Bh[kk][r] = __bfloat162float(Xhi[ib]);
            Bl[kk][r] = __bfloat162float(Xlo[ib]);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            float ah[4], al[4], bh[4], bl[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                ah[t] = Ah[kk][ty * 4 + t];
                al[t] = Al[kk][ty * 4 + t];
                bh[t] = Bh[kk][tx * 4 + t];
                bl[t] = Bl[kk][tx * 4 + t];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    acc[r][c] = fmaf(ah[r], bh[c], fmaf(ah[r], bl[c], fmaf(al[r], bh[c], acc[r][c])));
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int64_t gi = m0 + ty * 4 + r;
        if (gi >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t gc = c0 + tx * 4 + c;
            if (gc < ldu) U[gi * ldu + gc] = acc[r][c];
        }
    }
}

int gemm_3xbf16_simt(const wfq_geom *g, int64_t cpad, const __nv_bfloat16 *Xhi, const __nv_bfloat16 *Xlo, float *U,
                     int64_t ldu, cudaStream_t s) {
    // the X planes are read in 64-column tiles: cpad must cover them
    dim3 grid((unsigned)((ldu + 63) / 64), (unsigned)(g->npad / 64));
    KScope ks(g->ctx, WFQ_KT_GEMM_MIXED, s);
    k_gemm3_simt<<<grid, 256, 0, s>>>(g->n, g->npad, ldu, g->Dhi, g->Dlo, Xhi, Xlo, U); note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

}  // namespace wfq
