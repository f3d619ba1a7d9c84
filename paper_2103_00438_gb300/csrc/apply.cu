// Pieces of the operator apply y = (A - zI) x through the factored form of Eq. 17:
//   u = D x              (dense; FP64 stored / FP64 recomputed / 3xBF16 tensor cores)
//   y = Kbar u - P u - z x   (sparse neighbour term of Eq. 16-17 plus the shift of Eq. 14)
// Block vectors are atom-major: (atom i, complex column c) at i * cc + c.
#include "common.h"
#include "dfloat.cuh"

namespace wfq {

// ------------------------------------------------------------------ FP64 stored D: few columns

// U[i][:] = sum_k D[i][k] X[k][:] for C real columns (C <= 8): each warp owns 4 rows so
// that every X element read from L2 serves 4 D rows; D rows are read coalesced.
template <int C>
__global__ void __launch_bounds__(256) k_dgemv(int64_t n, const double *__restrict__ D,
                                               const double *__restrict__ X, double *__restrict__ U) {
    constexpr int RW = 4;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int64_t i0 = warp * RW;
    if (i0 >= n) return;
    double acc[RW][C];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = 0.0;
    const double *rows[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) rows[r] = D + min(i0 + r, n - 1) * n;
    int64_t k = lane;
    for (; k + 96 < n; k += 128) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int64_t kk = k + 32 * u;
            double x[C];
#pragma unroll
            for (int c = 0; c < C; ++c) x[c] = __ldg(X + kk * C + c);
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                double d = __ldcs(rows[r] + kk);
#pragma unroll
                for (int c = 0; c < C; ++c) acc[r][c] = fma(d, x[c], acc[r][c]);
            }
        }
    }
    for (; k < n; k += 32) {
        double x[C];
#pragma unroll
        for (int c = 0; c < C; ++c) x[c] = __ldg(X + k * C + c);
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            double d = __ldcs(rows[r] + k);
#pragma unroll
            for (int c = 0; c < C; ++c) acc[r][c] = fma(d, x[c], acc[r][c]);
        }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            double v = acc[r][c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[r][c] = v;
        }
    if (lane == 0) {
#pragma unroll
        for (int r = 0; r < RW; ++r)
            if (i0 + r < n)
#pragma unroll
                for (int c = 0; c < C; ++c) U[(i0 + r) * C + c] = acc[r][c];
    }
}

// ------------------------------------------------------------------ FP64 stored D: many columns

// U[n x C] = D[n x n] X[n x C], row-major, 64 x 64 tiles, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) k_dgemm(int64_t n, int64_t C, const double *__restrict__ D,
                                               const double *__restrict__ X, double *__restrict__ U) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < n; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            int e = tid + l * 256;
            int r = e >> 4, kk = e & 15;
            int64_t gi = m0 + r, gk = k0 + kk;
            As[kk][r] = (gi < n && gk < n) ? D[gi * n + gk] : 0.0;
            int kb = e >> 6, cb = e & 63;
            int64_t bk = k0 + kb, bc = n0 + cb;
            Bs[kb][cb] = (bk < n && bc < C) ? X[bk * C + bc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                a[t] = As[kk][ty * 4 + t];
                b[t] = Bs[kk][tx * 4 + t];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int64_t gi = m0 + ty * 4 + r;
        if (gi >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t gc = n0 + tx * 4 + c;
            if (gc < C) U[gi * C + gc] = acc[r][c];
        }
    }
}

// ------------------------------------------------------------------ FP64 matrix-free D

__device__ __forceinline__ double d_pair64(atom64_t a, atom64_t b) {
    double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    double r2 = dx * dx + dy * dy + dz * dz;
    double r = sqrt(r2);
    double s2 = a.w * a.w + b.w * b.w;
    if (r2 >= 36.0 * s2) return 1.0 / r;   // erf(r/sigma) == 1 in FP64 here
    return erf(r / sqrt(s2)) / r;
}

// As k_dgemm, with the D tile (Eq. 3) recomputed from the coordinates for every use.
__global__ void __launch_bounds__(256) k_dotf(int64_t n, int64_t C, const atom64_t *__restrict__ atom,
                                              const double *__restrict__ eta,
                                              const double *__restrict__ X, double *__restrict__ U) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][64];
    __shared__ atom64_t Ai[64];
    __shared__ double Ei[64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    if (tid < 64) {
        int64_t gi = min(m0 + tid, n - 1);
        Ai[tid] = atom[gi];
        Ei[tid] = eta[gi];
    }
    __syncthreads();
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < n; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            int e = tid + l * 256;
            int r = e & 63, kk = e >> 6;
            int64_t gi = m0 + r, gk = k0 + kk;
            double v = 0.0;
            if (gi < n && gk < n) v = (gi == gk) ? Ei[r] : d_pair64(Ai[r], atom[gk]);
            As[kk][r] = v;
            int kb = e >> 6, cb = e & 63;
            int64_t bk = k0 + kb, bc = n0 + cb;
            Bs[kb][cb] = (bk < n && bc < C) ? X[bk * C + bc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                a[t] = As[kk][ty * 4 + t];
                b[t] = Bs[kk][tx * 4 + t];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int64_t gi = m0 + ty * 4 + r;
        if (gi >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t gc = n0 + tx * 4 + c;
            if (gc < C) U[gi * C + gc] = acc[r][c];
        }
    }
}

// ------------------------------------------------------------------ double-float stored D

// U[n x C] = D[n x n] X[n x C] with double-float products (df_mac): every FP64 operand
// split into a float pair (hi = fp32(v), lo = fp32(v - hi): 48 significant bits).  This
// runs on the FP32 pipes, which GB300 has far more of than FP64.  PL: D comes from the
// stored FP32 pair planes (no FP64 arithmetic at all); else it is split from the FP64 D.

template <bool PL>
__global__ void __launch_bounds__(256) k_dgemm_df(int64_t n, int64_t C, const double *__restrict__ D,
                                                  const float *__restrict__ Fh, const float *__restrict__ Fl,
                                                  int64_t ldf, const double *__restrict__ X, double *__restrict__ U) {
    __shared__ float Ah[16][64], Al[16][64], Bh[16][64], Bl[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    float sh[4][4] = {}, sl[4][4] = {};
    for (int64_t k0 = 0; k0 < n; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = tid + l * 256;
            const int r = e >> 4, kk = e & 15;
            const int64_t gi = m0 + r, gk = k0 + kk;
            if (PL) {
                const bool in = gi < n && gk < n;
                Ah[kk][r] = in ? Fh[gi * ldf + gk] : 0.f;
                Al[kk][r] = in ? Fl[gi * ldf + gk] : 0.f;
            } else {
                df_split((gi < n && gk < n) ? D[gi * n + gk] : 0.0, Ah[kk][r], Al[kk][r]);
            }
            const int kb = e >> 6, cb = e & 63;
            const int64_t bk = k0 + kb, bc = n0 + cb;
            df_split((bk < n && bc < C) ? X[bk * C + bc] : 0.0, Bh[kb][cb], Bl[kb][cb]);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
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
                for (int c = 0; c < 4; ++c) df_mac(ah[r], al[r], bh[c], bl[c], sh[r][c], sl[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gi = m0 + ty * 4 + r;
        if (gi >= n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t gc = n0 + tx * 4 + c;
            if (gc < C) U[gi * C + gc] = (double)sh[r][c] + (double)sl[r][c];
        }
    }
}

// ------------------------------------------------------------------ double-float matrix-free D

// Exact a - b of two floats as an unevaluated sum (Knuth's two-difference).
__device__ __forceinline__ void two_diff(float a, float b, float &s, float &e) {
    s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fadd_rn(b, bb));
}

// (ah + al) - (bh + bl) as a normalised float pair.
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float &h, float &l) {
    float s, e;
    two_diff(ah, bh, s, e);
    e = __fadd_rn(e, __fsub_rn(al, bl));
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}

// (h + l)^2 accumulated into (sh, sl) with a two-sum.
__device__ __forceinline__ void df_sqr_acc(float h, float l, float &sh, float &sl) {
    const float p = __fmul_rn(h, h);
    const float e = fmaf(h, h, -p) + 2.0f * h * l;
    const float s = __fadd_rn(sh, p);
    const float v = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(p, v));
    sh = s;
    sl = sl + t + e;
}

// D_ik of Eq. 3 as a float pair.  Far pairs (r >= 6 sigma, where erf rounds to 1 in FP64):
// 1/r from the float-pair coordinates -- r^2 in double-float, FP32 rsqrt refined by one
// Newton step in double-float (relative error ~1e-13).  Near pairs and the diagonal: FP64.
__device__ __forceinline__ void d_pair_df_v(float4 pi0, float4 pi1, float4 pk0, float4 pk1,
                                            const atom64_t *__restrict__ a64, const double *__restrict__ eta,
                                            int64_t i, int64_t k, float &dh, float &dl) {
    if (i == k) {
        df_split(eta[i], dh, dl);
        return;
    }
    float xh, xl, yh, yl, zh, zl;
    df_sub(pi0.x, pi0.y, pk0.x, pk0.y, xh, xl);
    df_sub(pi0.z, pi0.w, pk0.z, pk0.w, yh, yl);
    df_sub(pi1.x, pi1.y, pk1.x, pk1.y, zh, zl);
    float rh = 0.f, rl = 0.f;
    df_sqr_acc(xh, xl, rh, rl);
    df_sqr_acc(yh, yl, rh, rl);
    df_sqr_acc(zh, zl, rh, rl);
    const float s2 = pi1.z * pi1.z + pk1.z * pk1.z;
    if (rh < 36.5f * s2) {   // near pair: FP64 (erf matters)
        df_split(d_pair64(a64[i], a64[k]), dh, dl);
        return;
    }
    const float y0 = rsqrtf(rh);
    const float th = __fmul_rn(y0, y0);
    const float tl = fmaf(y0, y0, -th);
    const float uh = __fmul_rn(rh, th);
    const float ul = fmaf(rh, th, -uh) + rh * tl + rl * th;
    const float delta = __fsub_rn(1.0f, uh) - ul;   // 1 - r^2 y0^2, ~1e-7
    dh = y0;
    dl = 0.5f * y0 * delta;
}

__device__ __forceinline__ void d_pair_df(const float4 *__restrict__ adf, const atom64_t *__restrict__ a64,
                                          const double *__restrict__ eta, int64_t i, int64_t k, float &dh,
                                          float &dl) {
    // (xh, xl, yh, yl), (zh, zl, w, -) float pairs per atom
    d_pair_df_v(adf[2 * i], adf[2 * i + 1], adf[2 * k], adf[2 * k + 1], a64, eta, i, k, dh, dl);
}

// U[d][i] = sum_j D_ij x[d][j] for C <= 4 real vectors (direction-major, float-pair split
// xh / xl), with D generated as float pairs from the coordinates (d_pair_df) -- the
// matrix-free form of the shifted solver's product.  A warp owns MFV_ROWS rows; its lanes
// walk the columns, each column's atom record and x loaded once for all the warp's rows.
constexpr int MFV_ROWS = 2;
template <int C>
__global__ void __launch_bounds__(256) k_dotf_dfv(int64_t n, const float4 *__restrict__ adf,
                                                  const atom64_t *__restrict__ a64, const double *__restrict__ eta,
                                                  const float *__restrict__ xh, const float *__restrict__ xl,
                                                  double *__restrict__ U) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = ((int64_t)blockIdx.x * 8 + warp) * MFV_ROWS;
    float4 pi0[MFV_ROWS], pi1[MFV_ROWS];
    float sh[MFV_ROWS][C], sl[MFV_ROWS][C];
#pragma unroll
    for (int r = 0; r < MFV_ROWS; ++r) {
        const int64_t i = row0 + r < n ? row0 + r : n - 1;   // rows past n compute, never store
        pi0[r] = adf[2 * i];
        pi1[r] = adf[2 * i + 1];
#pragma unroll
        for (int d = 0; d < C; ++d) sh[r][d] = sl[r][d] = 0.f;
    }
    for (int64_t k = lane; k < n; k += 32) {
        const float4 pk0 = adf[2 * k], pk1 = adf[2 * k + 1];
        float xkh[C], xkl[C];
#pragma unroll
        for (int d = 0; d < C; ++d) {
            xkh[d] = xh[(int64_t)d * n + k];
            xkl[d] = xl[(int64_t)d * n + k];
        }
#pragma unroll
        for (int r = 0; r < MFV_ROWS; ++r) {
            const int64_t i = row0 + r < n ? row0 + r : n - 1;
            float dh, dl;
            d_pair_df_v(pi0[r], pi1[r], pk0, pk1, a64, eta, i, k, dh, dl);
#pragma unroll
            for (int d = 0; d < C; ++d) df_mac(dh, dl, xkh[d], xkl[d], sh[r][d], sl[r][d]);
        }
    }
#pragma unroll
    for (int r = 0; r < MFV_ROWS; ++r)
#pragma unroll
        for (int d = 0; d < C; ++d)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, sh[r][d], off);
                const float ol = __shfl_xor_sync(0xffffffffu, sl[r][d], off);
                df_add(sh[r][d], sl[r][d], oh, ol);
            }
    if (lane == 0)
#pragma unroll
        for (int r = 0; r < MFV_ROWS; ++r)
            if (row0 + r < n)
#pragma unroll
                for (int d = 0; d < C; ++d) U[(int64_t)d * n + row0 + r] = (double)sh[r][d] + (double)sl[r][d];
}

// A BEM geometry stores its operator; the kernels that regenerate D from the coordinates
// (Eq. 3) must never see one.
static int require_wfq(const wfq_geom *g) {
    if (g->op != OP_WFQ)
        return fail(WFQ_EUNSUPPORTED, "matrix-free products regenerate the omega-FQ D; a BEM geometry stores its operator");
    return WFQ_OK;
}

int d_gemv_df_mf(const wfq_geom *g, int C, const float *xh, const float *xl, double *U, cudaStream_t s) {
    WFQ_TRY(require_wfq(g));
    const int64_t n = g->n;
    const unsigned blocks = (unsigned)((n + 8 * MFV_ROWS - 1) / (8 * MFV_ROWS));
    switch (C) {
        case 1: k_dotf_dfv<1><<<blocks, 256, 0, s>>>(n, g->atomdf, g->atom64, g->eta, xh, xl, U); break;
        case 2: k_dotf_dfv<2><<<blocks, 256, 0, s>>>(n, g->atomdf, g->atom64, g->eta, xh, xl, U); break;
        case 3: k_dotf_dfv<3><<<blocks, 256, 0, s>>>(n, g->atomdf, g->atom64, g->eta, xh, xl, U); break;
        default: k_dotf_dfv<4><<<blocks, 256, 0, s>>>(n, g->atomdf, g->atom64, g->eta, xh, xl, U); break;
    }
    note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

// As k_dgemm_df with the D tile generated per use (matrix-free); TN columns per thread.
template <int TN>
__global__ void __launch_bounds__(256) k_dotf_df(int64_t n, int64_t C, const float4 *__restrict__ adf,
                                                 const atom64_t *__restrict__ a64, const double *__restrict__ eta,
                                                 const double *__restrict__ X, double *__restrict__ U) {
    constexpr int BN = 16 * TN;
    __shared__ float Ah[16][64], Al[16][64], Bh[16][BN], Bl[16][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * BN;
    float sh[4][TN] = {}, sl[4][TN] = {};
    for (int64_t k0 = 0; k0 < n; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = tid + l * 256;
            const int r = e & 63, kk = e >> 6;
            const int64_t gi = m0 + r, gk = k0 + kk;
            float h = 0.f, lo = 0.f;
            if (gi < n && gk < n) d_pair_df(adf, a64, eta, gi, gk, h, lo);
            Ah[kk][r] = h;
            Al[kk][r] = lo;
        }
        for (int e = tid; e < 16 * BN; e += 256) {
            const int kb = e / BN, cb = e % BN;
            const int64_t bk = k0 + kb, bc = n0 + cb;
            df_split((bk < n && bc < C) ? X[bk * C + bc] : 0.0, Bh[kb][cb], Bl[kb][cb]);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            float ah[4], al[4], bh[TN], bl[TN];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                ah[t] = Ah[kk][ty * 4 + t];
                al[t] = Al[kk][ty * 4 + t];
            }
#pragma unroll
            for (int t = 0; t < TN; ++t) {
                bh[t] = Bh[kk][tx * TN + t];
                bl[t] = Bl[kk][tx * TN + t];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) df_mac(ah[r], al[r], bh[c], bl[c], sh[r][c], sl[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gi = m0 + ty * 4 + r;
        if (gi >= n) continue;
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int64_t gc = n0 + tx * TN + c;
            if (gc < C) U[gi * C + gc] = (double)sh[r][c] + (double)sl[r][c];
        }
    }
}

int d_apply_df(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s) {
    // symmetric float-pair tiles: read them, 4 real vectors per pass (the product that
    // regenerates D from the coordinates' float pairs held the true residual of a 1.5e5-atom
    // sodium sphere near 5e-7, where the stored pairs reach 5e-9)
    if (!g->D64 && !g->Dfh && g->Dsym) return d_apply_pairs_df(g, cc, X, U, s);
    if (!g->D64 && !g->Dfh) {
        // matrix-free double-float product
        WFQ_TRY(require_wfq(g));
        const int64_t n = g->n, C = 2 * cc;
        // few columns: the double-float GEMV that regenerates D per product (the shifted
        // solver's matrix-free product, up to 4 real vectors per launch)
        if (C <= 8) return d_apply_mf_gemv_df(g, cc, X, U, s);
        KScope ks(g->ctx, WFQ_KT_DAPPLY_FP64, s, 2.0 * (double)n * (double)n * (double)C);
        const double *x = reinterpret_cast<const double *>(X);
        double *u = reinterpret_cast<double *>(U);
        if (C <= 32) {
            dim3 grid((unsigned)((C + 31) / 32), (unsigned)((n + 63) / 64));
            if (grid.y > 65535u) return fail(WFQ_EUNSUPPORTED, "double-float apply: too many rows");
            k_dotf_df<2><<<grid, 256, 0, s>>>(n, C, g->atomdf, g->atom64, g->eta, x, u); note_launch();
        } else {
            dim3 grid((unsigned)((C + 63) / 64), (unsigned)((n + 63) / 64));
            if (grid.y > 65535u) return fail(WFQ_EUNSUPPORTED, "double-float apply: too many rows");
            k_dotf_df<4><<<grid, 256, 0, s>>>(n, C, g->atomdf, g->atom64, g->eta, x, u); note_launch();
        }
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }
    const int64_t n = g->n, C = 2 * cc;
    if (C <= 8 && g->D64) return d_apply_fp64(g, cc, X, U, s);   // few columns: memory bound, FP64 GEMV
    KScope ks(g->ctx, WFQ_KT_DAPPLY_FP64, s, 2.0 * (double)n * (double)n * (double)C);
    dim3 grid((unsigned)((C + 63) / 64), (unsigned)((n + 63) / 64));
    if (grid.y > 65535u) return fail(WFQ_EUNSUPPORTED, "double-float apply: too many rows");
    const double *x = reinterpret_cast<const double *>(X);
    double *u = reinterpret_cast<double *>(U);
    if (g->Dfh)
        k_dgemm_df<true><<<grid, 256, 0, s>>>(n, C, nullptr, g->Dfh, g->Dfl, g->ldf, x, u);
    else
        k_dgemm_df<false><<<grid, 256, 0, s>>>(n, C, g->D64, nullptr, nullptr, 0, x, u);
    note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

int d_apply_fp64(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s) {
    const int64_t n = g->n, C = 2 * cc;
    // no FP64 D but stored float pairs: their double-float product (2^-48 per product, on
    // the FP32 pipes and at 8 or 4 bytes per entry) instead of regenerating D in FP64
    if (!g->D64 && (g->Dfh || g->Dsym) && C <= 8) return d_apply_pairs_df(g, cc, X, U, s);
    const double *x = reinterpret_cast<const double *>(X);
    double *u = reinterpret_cast<double *>(U);
    KScope ks(g->ctx, WFQ_KT_DAPPLY_FP64, s, 2.0 * (double)n * (double)n * (double)C);
    if (g->D64 && C <= 8) {
        int64_t warps = (n + 3) / 4;
        unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
        switch (C) {
            case 2: k_dgemv<2><<<blocks, 256, 0, s>>>(n, g->D64, x, u); note_launch(); break;
            case 4: k_dgemv<4><<<blocks, 256, 0, s>>>(n, g->D64, x, u); note_launch(); break;
            case 6: k_dgemv<6><<<blocks, 256, 0, s>>>(n, g->D64, x, u); note_launch(); break;
            default: k_dgemv<8><<<blocks, 256, 0, s>>>(n, g->D64, x, u); note_launch(); break;
        }
    } else {
        dim3 grid((unsigned)((C + 63) / 64), (unsigned)((n + 63) / 64));
        if (grid.y > 65535u) return fail(WFQ_EUNSUPPORTED, "FP64 apply: too many rows");
        if (g->D64) {
            k_dgemm<<<grid, 256, 0, s>>>(n, C, g->D64, x, u);
        } else {
            WFQ_TRY(require_wfq(g));
            k_dotf<<<grid, 256, 0, s>>>(n, C, g->atom64, g->eta, x, u);
        }
        note_launch();
    }
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

// ------------------------------------------------------------------ sparse term + shift

template <class V>
struct CplxT;
template <>
struct CplxT<double2> {
    using R = double;
};
template <>
struct CplxT<float2> {
    using R = float;
};

// Many columns: one warp per atom row, lanes over complex columns.
// Y_i = sum_p Kbar_ip (U_j - U_i) - z X_i  (the difference form of Kbar U - P U).
template <class V, class VAL>
__global__ void __launch_bounds__(128) k_sparse_cols(int64_t n, int64_t cc,
                                                     const int64_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ col,
                                                     const VAL *__restrict__ val,
                                                     const V *__restrict__ U, const V *__restrict__ X,
                                                     const double2 *__restrict__ z, V *__restrict__ Y) {
    using R = typename CplxT<V>::R;
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t p0 = rowptr[i], p1 = rowptr[i + 1];
    for (int64_t c = lane; c < cc; c += 32) {
        V ui = U[i * cc + c];
        R ax = 0, ay = 0;
        for (int64_t p = p0; p < p1; ++p) {
            R w = (R)val[p];
            V uj = U[(int64_t)col[p] * cc + c];
            ax += w * (uj.x - ui.x);
            ay += w * (uj.y - ui.y);
        }
        V xv = X[i * cc + c];
        double2 zc = z[c];
        R zr = (R)zc.x, zi = (R)zc.y;
        V out;
        out.x = ax - (zr * xv.x - zi * xv.y);
        out.y = ay - (zr * xv.y + zi * xv.x);
        Y[i * cc + c] = out;
    }
}

// Few columns (cc <= 4): one warp per atom row, lanes over neighbours.
template <class V, class VAL, int CC>
__global__ void __launch_bounds__(128) k_sparse_nbrs(int64_t n, const int64_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ col,
                                                     const VAL *__restrict__ val,
                                                     const V *__restrict__ U, const V *__restrict__ X,
                                                     const double2 *__restrict__ z, V *__restrict__ Y) {
    using R = typename CplxT<V>::R;
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t p0 = rowptr[i], p1 = rowptr[i + 1];
    V ui[CC];
    R ax[CC], ay[CC];
#pragma unroll
    for (int c = 0; c < CC; ++c) {
        ui[c] = U[i * CC + c];
        ax[c] = 0;
        ay[c] = 0;
    }
    for (int64_t p = p0 + lane; p < p1; p += 32) {
        R w = (R)val[p];
        int64_t j = col[p];
#pragma unroll
        for (int c = 0; c < CC; ++c) {
            V uj = U[j * CC + c];
            ax[c] += w * (uj.x - ui[c].x);
            ay[c] += w * (uj.y - ui[c].y);
        }
    }
#pragma unroll
    for (int c = 0; c < CC; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ax[c] += __shfl_xor_sync(0xffffffffu, ax[c], o);
            ay[c] += __shfl_xor_sync(0xffffffffu, ay[c], o);
        }
    }
    if (lane < CC) {
        // lane c writes column c
#pragma unroll
        for (int c = 0; c < CC; ++c) {
            if (c != lane) continue;
            V xv = X[i * CC + c];
            double2 zc = z[c];
            R zr = (R)zc.x, zi = (R)zc.y;
            V out;
            out.x = ax[c] - (zr * xv.x - zi * xv.y);
            out.y = ay[c] - (zr * xv.y + zi * xv.x);
            Y[i * CC + c] = out;
        }
    }
}

// BEM geometries (no sparse term): Y = U - z_c X elementwise, column c = e % cc.
template <class V>
__global__ void __launch_bounds__(256) k_shift_only(int64_t total, int64_t cc, const V *__restrict__ U,
                                                    const V *__restrict__ X, const double2 *__restrict__ z,
                                                    V *__restrict__ Y) {
    using R = typename CplxT<V>::R;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const double2 zc = z[e % cc];
    const R zr = (R)zc.x, zi = (R)zc.y;
    const V u = U[e], xv = X[e];
    V out;
    out.x = u.x - (zr * xv.x - zi * xv.y);
    out.y = u.y - (zr * xv.y + zi * xv.x);
    Y[e] = out;
}

template <class V, class VAL>
static int sparse_shift_impl(const wfq_geom *g, int64_t cc, const V *U, const V *X, const double2 *z,
                             V *Y, const VAL *val, cudaStream_t s) {
    const int64_t n = g->n;
    unsigned blocks = (unsigned)((n * 32 + 127) / 128);
    KScope ks(g->ctx, WFQ_KT_SPARSE, s);
    if (g->op == OP_BEM) {
        const int64_t total = n * cc;
        k_shift_only<V><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, cc, U, X, z, Y); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }
    switch (cc) {
        case 1: k_sparse_nbrs<V, VAL, 1><<<blocks, 128, 0, s>>>(n, g->rowptr, g->col, val, U, X, z, Y); note_launch(); break;
        case 2: k_sparse_nbrs<V, VAL, 2><<<blocks, 128, 0, s>>>(n, g->rowptr, g->col, val, U, X, z, Y); note_launch(); break;
        case 3: k_sparse_nbrs<V, VAL, 3><<<blocks, 128, 0, s>>>(n, g->rowptr, g->col, val, U, X, z, Y); note_launch(); break;
        case 4: k_sparse_nbrs<V, VAL, 4><<<blocks, 128, 0, s>>>(n, g->rowptr, g->col, val, U, X, z, Y); note_launch(); break;
        default:
            k_sparse_cols<V, VAL><<<blocks, 128, 0, s>>>(n, cc, g->rowptr, g->col, val, U, X, z, Y); note_launch();
    }
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

int sparse_shift_fp64(const wfq_geom *g, int64_t cc, const double2 *U, const double2 *X,
                      const double2 *z, double2 *Y, cudaStream_t s) {
    return sparse_shift_impl<double2, double>(g, cc, U, X, z, Y, g->val64, s);
}

int sparse_shift_fp32(const wfq_geom *g, int64_t cc, const float2 *U, const float2 *X,
                      const double2 *z, float2 *Y, cudaStream_t s) {
    return sparse_shift_impl<float2, float>(g, cc, U, X, z, Y, g->val32, s);
}

// ------------------------------------------------------------------ mixed: split + GEMM

// X: n x (2 cc) real view (complex64 atom-major) -> Xhi/Xlo: [cpad][npad] bf16 (K-major
// operand of the GEMM), hi = bf16(x), lo = bf16(x - hi); zero padding.
__global__ void __launch_bounds__(256) k_split_bf16(int64_t n, int64_t npad, int64_t C, int64_t cpad,
                                                    const float *__restrict__ X,
                                                    __nv_bfloat16 *__restrict__ hi,
                                                    __nv_bfloat16 *__restrict__ lo) {
    __shared__ float t[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t a0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        int64_t a = a0 + r, c = c0 + tx;
        t[r][tx] = (a < n && c < C) ? X[a * C + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        int64_t c = c0 + r, a = a0 + tx;
        if (c < cpad && a < npad) {
            float v = t[tx][r];
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            hi[c * npad + a] = h;
            lo[c * npad + a] = l;
        }
    }
}

// Rows of the bf16 X planes: the real columns rounded up to 32 (the accumulator is read
// back from tensor memory in 32-column chunks; MMA N is a multiple of 16).
static int64_t mixed_cpad(int64_t cc) { return round_up(2 * cc, 32); }

size_t mixed_scratch_bytes(const wfq_geom *g, int64_t cc) {
    int64_t cpad = mixed_cpad(cc);
    return (size_t)2 * cpad * g->npad * sizeof(__nv_bfloat16);
}

int d_apply_mixed(const wfq_geom *g, int64_t cc, const float2 *X, float2 *U, void *scratch,
                  cudaStream_t s) {
    // without stored planes, the fast-multipole product when its tree is built (at large N
    // both faster and, at order >= 6, closer to D than the generated 3xBF16 tiles)
    if (!g->Dhi && g->fmm && cc <= 256) return d_apply_fmm(g, cc, X, U, s);
    if (!g->Dhi) WFQ_TRY(require_wfq(g));
    const int64_t C = 2 * cc, cpad = mixed_cpad(cc), npad = g->npad;
    __nv_bfloat16 *xhi = reinterpret_cast<__nv_bfloat16 *>(scratch);
    __nv_bfloat16 *xlo = xhi + cpad * npad;
    dim3 grid((unsigned)(npad / 32), (unsigned)((cpad + 31) / 32));
    k_split_bf16<<<grid, 256, 0, s>>>(g->n, npad, C, cpad, reinterpret_cast<const float *>(X), xhi, xlo); note_launch();
    WFQ_CUDA(cudaGetLastError());
    if (g->Dhi) return gemm_3xbf16(g, cpad, xhi, xlo, reinterpret_cast<float *>(U), C, s);
    return gemm_3xbf16_mf(g, cpad, xhi, xlo, reinterpret_cast<float *>(U), C, s);
}

}  // namespace wfq
