// Shifted GMRES: one real Arnoldi process per field direction serves every frequency.
//
// A = (Kbar - P) D and the right-hand sides R_k are real and do not depend on omega
// (Section 2.1, Eq. 13-14); only the shift z(omega) of Eq. 12 does.  Hence the Krylov
// space K_j(A - z I, R_k) equals K_j(A, R_k) for every z, and one Arnoldi process on A
// (Eq. 24's basis, started from R_k, real arithmetic) gives for all shifts at once
//
//     A V_j = V_{j+1} Hbar_j    =>    (A - z I) V_j = V_{j+1} (Hbar_j - z Ibar_j),
//
// with Ibar_j the (j+1) x j identity.  The GMRES iterate of column (omega, k) from x0 = 0
// is x = V_j y with y minimising || ||R_k|| e1 - (Hbar_j - z Ibar_j) y ||, which each
// column solves by its own complex Givens QR of the shared real Hbar_j.  One D product of
// the ndir real Arnoldi vectors per iteration therefore serves all nfreq x ndir columns.
//
// Precision: the Arnoldi vectors, Hbar and the rotations are FP64; D is applied with
// double-float products (~2^-48 relative) on the FP32 pipes, from the stored FP32 pair
// planes (or split from the FP64 D).  Every column's true residual R - (A - zI) q is
// measured at the end in FP64 from q = sum_k v_k y_k and D q = sum_k (D v_k) y_k, the D
// products of the Arnoldi vectors kept from the iteration (D is linear, so this is D q up
// to the rounding of the double-float products; neither Hbar nor the orthogonality of the
// basis enters).  Columns above the tolerance (the basis reached its cap, or rounding of
// the shared process) continue from their iterate in the block GMRES(m) solver.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"
#include "dfloat.cuh"

namespace wfq {
namespace {

inline unsigned nblk(int64_t total, int t = 256) { return (unsigned)((total + t - 1) / t); }

// Threads per block of the one-thread-per-column Givens step: its work is a serial FP64
// chain per column, and GB300 has only about two FP64 FMAs per clock per SM, so the columns
// are spread over many SMs instead of filling one.
constexpr int PER_COLUMN_BLOCK = 4;

__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_scale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_conjmul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double c_abs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 c_div(double2 a, double2 b) {
    const double d = c_abs2(b);
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ------------------------------------------------------------------ operator: A v (real)

// Tilings of the double-float GEMV: rows per warp, 128-column load steps in flight per lane,
// resident blocks per SM the register budget must allow.  The kernel is bound by
// instruction issue of the double-float arithmetic (~12 FP32 instructions per entry and
// vector) as much as by memory; which tiling overlaps the two best depends on N and on the
// number of vectors, so the first product of each shape times all of them on the real
// operands and keeps the fastest (autotune below).  A sweep at N = 20000 found 0.75-0.85 ms
// per launch for these four and 0.9-1.4 ms for wider or 16-warp tilings.  Staging x by
// asynchronous copies into two 512-column buffers, with each chunk's first D loads issued
// ahead of the barrier, measured slower (0.728 vs 0.679 ms per cnt20k product); so did
// streaming D through shared memory by 2-D bulk tensor copies (a producer lane, a 4-stage
// mbarrier ring of 8 or 16 rows x 256 columns, 8 consumer warps, 2 CTAs per SM): 2.24 and
// 1.43 ms per cnt20k product.
constexpr int GV_WARPS = 8;      // warps per block
constexpr int GV_CHUNK = 1024;   // x entries staged in shared memory per step
constexpr int GV_NTILINGS = 4;

// U[d][i] = sum_j D_ij x[d][j] for C real vectors (direction-major, length n), with
// double-float products.  Each warp owns ROWS rows and reads them with 16-byte loads
// (four consecutive j per lane), TB steps of 128 columns at a time so that 2 * ROWS * TB
// independent loads per lane are in flight before any is used; x is staged per
// chunk in shared memory as separate hi / lo planes so that a quarter-warp's 16-byte reads
// are conflict-free.  PL: D from the FP32 pair planes (row pitch ld, a multiple of 4, zero
// beyond n); else split from the FP64 D.  Entries past n contribute zero (x is zero there).
template <int C, bool PL, int ROWS, int TB, int MINB>
__global__ void __launch_bounds__(GV_WARPS * 32, MINB) k_dgemv_df(int64_t n, int64_t ld, const float *__restrict__ Fh,
                                                            const float *__restrict__ Fl,
                                                            const double *__restrict__ D64,
                                                            const float *__restrict__ xh,
                                                            const float *__restrict__ xl, double *__restrict__ U) {
    __shared__ __align__(16) float sxh[C][GV_CHUNK];
    __shared__ __align__(16) float sxl[C][GV_CHUNK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = ((int64_t)blockIdx.x * GV_WARPS + warp) * ROWS;
    // FP32 planes (PL): rows of ld floats, ld a multiple of 128, zero past column n, so a
    // 128-column step that starts below n lies inside the row and needs no column check;
    // rows past n read the last row (their results are dropped).  This lane's float4 of
    // each row, as a pointer advanced by the step's float4 index.
    const float4 *rowh[ROWS], *rowl[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        if constexpr (PL) {
            const int64_t i = row0 + r, ic = i < n ? i : n - 1;
            rowh[r] = reinterpret_cast<const float4 *>(Fh + ic * ld) + lane;
            rowl[r] = reinterpret_cast<const float4 *>(Fl + ic * ld) + lane;
        } else {
            rowh[r] = rowl[r] = nullptr;
        }
    }
    // accumulators per (row, vector): even and odd columns in the two lanes of a float2
    float2 sh2[ROWS][C], sl2[ROWS][C];
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int d = 0; d < C; ++d) sh2[r][d] = sl2[r][d] = make_float2(0.f, 0.f);

    for (int64_t j0 = 0; j0 < n; j0 += GV_CHUNK) {
        __syncthreads();
        for (int t = threadIdx.x; t < C * GV_CHUNK; t += GV_WARPS * 32) {
            const int d = t / GV_CHUNK, jj = t - d * GV_CHUNK;
            const int64_t j = j0 + jj;
            sxh[d][jj] = j < n ? xh[(int64_t)d * n + j] : 0.f;
            sxl[d][jj] = j < n ? xl[(int64_t)d * n + j] : 0.f;
        }
        __syncthreads();
        const int64_t trem = (n - j0 + 127) / 128;
        const int tend = trem < GV_CHUNK / 128 ? (int)trem : GV_CHUNK / 128;
        for (int t0 = 0; t0 < tend; t0 += TB) {
            float4 dh[TB][ROWS], dl[TB][ROWS];
#pragma unroll
            for (int t = 0; t < TB; ++t) {
                const int tt = t0 + t;
                const int64_t j = j0 + tt * 128 + lane * 4;
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const int64_t i = row0 + r;
                    if constexpr (PL) {
                        if (tt < tend) {   // warp-uniform: the last chunk may end inside the TB group
                            const int64_t q = (j0 >> 2) + tt * 32;
                            dh[t][r] = __ldg(rowh[r] + q);
                            dl[t][r] = __ldg(rowl[r] + q);
                        } else {
                            dh[t][r] = dl[t][r] = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    } else if (i >= n || j >= n) {
                        dh[t][r] = dl[t][r] = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        const double *row = D64 + i * n;
                        float h[4], l[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) df_split(j + e < n ? __ldg(row + j + e) : 0.0, h[e], l[e]);
                        dh[t][r] = make_float4(h[0], h[1], h[2], h[3]);
                        dl[t][r] = make_float4(l[0], l[1], l[2], l[3]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < TB; ++t) {
                const int jl = (t0 + t) * 128 + lane * 4;
#pragma unroll
                for (int d = 0; d < C; ++d) {
                    const float4 xh4 = *reinterpret_cast<const float4 *>(&sxh[d][jl]);
                    const float4 xl4 = *reinterpret_cast<const float4 *>(&sxl[d][jl]);
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        df_mac2(make_float2(dh[t][r].x, dh[t][r].y), make_float2(dl[t][r].x, dl[t][r].y),
                                make_float2(xh4.x, xh4.y), make_float2(xl4.x, xl4.y), sh2[r][d], sl2[r][d]);
                        df_mac2(make_float2(dh[t][r].z, dh[t][r].w), make_float2(dl[t][r].z, dl[t][r].w),
                                make_float2(xh4.z, xh4.w), make_float2(xl4.z, xl4.w), sh2[r][d], sl2[r][d]);
                    }
                }
            }
        }
    }
    // the two lanes, then warp sums in double-float, fixed butterfly order
    float sh[ROWS][C], sl[ROWS][C];
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int d = 0; d < C; ++d) {
            sh[r][d] = sh2[r][d].x;
            sl[r][d] = sl2[r][d].x;
            df_add(sh[r][d], sl[r][d], sh2[r][d].y, sl2[r][d].y);
        }
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int d = 0; d < C; ++d)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, sh[r][d], off);
                const float ol = __shfl_xor_sync(0xffffffffu, sl[r][d], off);
                df_add(sh[r][d], sl[r][d], oh, ol);
            }
    if (lane == 0) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int64_t i = row0 + r;
            if (i < n)
#pragma unroll
                for (int d = 0; d < C; ++d) U[(int64_t)d * n + i] = (double)sh[r][d] + (double)sl[r][d];
        }
    }
}

// ---- the same product from the symmetric tiled storage (upper-triangle 64 x 64 tiles):
// every stored tile (I, J), I < J, serves both U_I += D_IJ x_J and U_J += D_IJ^T x_I, so D is
// read once for the triangle instead of the full matrix -- half the memory; the time is
// that of the full-plane product (both are bound by issue of the double-float arithmetic:
// 0.76 vs 0.74 ms at N = 20000).  One CTA per work item (tiles J0 ..
// J1 - 1 of tile row I); thread (tr, tc) of the 16 x 16 grid owns a 4 x 4 sub-block of each
// tile.  Row sums accumulate over the item in registers; the column sums of a tile are
// reduced over the 16 thread rows in shared memory.  Both go out as float pairs (rowpart per
// item, colpart per tile) and k_dsymv_finish adds them up in a fixed order.  The diagonal
// tile, stored in full, contributes only row sums.
constexpr int SY_T = (int)kSymTile;

template <int C>
__global__ void __launch_bounds__(256, 2) k_dsymv_df(int64_t n, int64_t T, const float *__restrict__ Dsym,
                                                     const SymItem *__restrict__ items,
                                                     const float *__restrict__ xh, const float *__restrict__ xl,
                                                     float2 *__restrict__ rowpart, float2 *__restrict__ colpart) {
    __shared__ __align__(16) float sxh[C][SY_T];
    __shared__ __align__(16) float sxl[C][SY_T];
    __shared__ float2 cred[16][SY_T * C];
    const SymItem it = items[blockIdx.x];
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    const int64_t I = it.I;
    float xih[4][C], xil[4][C], rh[4][C], rl[4][C];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = I * SY_T + tr * 4 + r;
#pragma unroll
        for (int d = 0; d < C; ++d) {
            xih[r][d] = i < n ? xh[(int64_t)d * n + i] : 0.f;
            xil[r][d] = i < n ? xl[(int64_t)d * n + i] : 0.f;
            rh[r][d] = rl[r][d] = 0.f;
        }
    }
    for (int J = it.J0; J < it.J1; ++J) {
        const int64_t t = sym_tile(I, J, T);
        const float *th = Dsym + t * 2 * SY_T * SY_T, *tl = th + SY_T * SY_T;
        __syncthreads();   // the previous tile's shared-memory readers are done
        if (tid < C * SY_T) {
            const int d = tid / SY_T, c = tid % SY_T;
            const int64_t j = (int64_t)J * SY_T + c;
            sxh[d][c] = j < n ? xh[(int64_t)d * n + j] : 0.f;
            sxl[d][c] = j < n ? xl[(int64_t)d * n + j] : 0.f;
        }
        float4 dh[4], dl[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            dh[r] = __ldg(reinterpret_cast<const float4 *>(th + (tr * 4 + r) * SY_T + tc * 4));
            dl[r] = __ldg(reinterpret_cast<const float4 *>(tl + (tr * 4 + r) * SY_T + tc * 4));
        }
        __syncthreads();
        const bool diag = J == I;
        float ch[4][C], cl[4][C];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int d = 0; d < C; ++d) ch[c][d] = cl[c][d] = 0.f;
#pragma unroll
        for (int d = 0; d < C; ++d) {
            const float4 ah = *reinterpret_cast<const float4 *>(&sxh[d][tc * 4]);
            const float4 al = *reinterpret_cast<const float4 *>(&sxl[d][tc * 4]);
            const float xjh[4] = {ah.x, ah.y, ah.z, ah.w}, xjl[4] = {al.x, al.y, al.z, al.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float vh[4] = {dh[r].x, dh[r].y, dh[r].z, dh[r].w};
                const float vl[4] = {dl[r].x, dl[r].y, dl[r].z, dl[r].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    df_mac(vh[c], vl[c], xjh[c], xjl[c], rh[r][d], rl[r][d]);
                    if (!diag) df_mac(vh[c], vl[c], xih[r][d], xil[r][d], ch[c][d], cl[c][d]);
                }
            }
        }
        if (!diag) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int d = 0; d < C; ++d) cred[tr][(tc * 4 + c) * C + d] = make_float2(ch[c][d], cl[c][d]);
            __syncthreads();
            if (tid < SY_T * C) {
                float sh = 0.f, sl = 0.f;
#pragma unroll
                for (int q = 0; q < 16; ++q) df_add(sh, sl, cred[q][tid].x, cred[q][tid].y);
                colpart[t * SY_T * C + tid] = make_float2(sh, sl);   // (column, direction) = (tid / C, tid % C)
            }
        }
    }
    // row sums over the 16 threads of a thread row (16 consecutive lanes), fixed butterfly
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int d = 0; d < C; ++d)
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, rh[r][d], off);
                const float ol = __shfl_xor_sync(0xffffffffu, rl[r][d], off);
                df_add(rh[r][d], rl[r][d], oh, ol);
            }
    if (tc == 0)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int d = 0; d < C; ++d)
                rowpart[((int64_t)blockIdx.x * SY_T + tr * 4 + r) * C + d] = make_float2(rh[r][d], rl[r][d]);
}

// U[d][i] = (row sums of the items of tile row K) + (column sums of tiles (I, K), I < K),
// K = i / 64, added in that fixed order in double-float.
__global__ void k_dsymv_finish(int64_t n, int C, int64_t T, const int *__restrict__ item_start,
                               const float2 *__restrict__ rowpart, const float2 *__restrict__ colpart,
                               double *__restrict__ U) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * C) return;
    const int d = (int)(e / n);
    const int64_t i = e - (int64_t)d * n, K = i / SY_T, r = i % SY_T;
    float sh = 0.f, sl = 0.f;
    for (int q = item_start[K]; q < item_start[K + 1]; ++q) {
        const float2 v = rowpart[((int64_t)q * SY_T + r) * C + d];
        df_add(sh, sl, v.x, v.y);
    }
    for (int64_t I = 0; I < K; ++I) {
        const float2 v = colpart[(sym_tile(I, K, T) * SY_T + r) * C + d];
        df_add(sh, sl, v.x, v.y);
    }
    U[e] = (double)sh + (double)sl;
}

template <int C, bool PL>
void launch_dgemv(int tiling, int64_t n, int64_t ld, const float *Fh, const float *Fl, const double *D64,
                  const float *xh, const float *xl, double *U, cudaStream_t s) {
    const unsigned b1 = (unsigned)((n + GV_WARPS - 1) / GV_WARPS), b2 = (unsigned)((n + 2 * GV_WARPS - 1) / (2 * GV_WARPS));
    switch (tiling) {
        case 1: k_dgemv_df<C, PL, 2, 4, 2><<<b2, GV_WARPS * 32, 0, s>>>(n, ld, Fh, Fl, D64, xh, xl, U); break;
        case 2: k_dgemv_df<C, PL, 2, 2, 3><<<b2, GV_WARPS * 32, 0, s>>>(n, ld, Fh, Fl, D64, xh, xl, U); break;
        case 3: k_dgemv_df<C, PL, 1, 8, 2><<<b1, GV_WARPS * 32, 0, s>>>(n, ld, Fh, Fl, D64, xh, xl, U); break;
        default: k_dgemv_df<C, PL, 1, 4, 3><<<b1, GV_WARPS * 32, 0, s>>>(n, ld, Fh, Fl, D64, xh, xl, U); break;
    }
}

template <bool PL>
void launch_dgemv_c(int cg, int tiling, int64_t n, int64_t ld, const float *Fh, const float *Fl, const double *D64,
                    const float *xh, const float *xl, double *U, cudaStream_t s) {
    switch (cg) {
        case 1: launch_dgemv<1, PL>(tiling, n, ld, Fh, Fl, D64, xh, xl, U, s); break;
        case 2: launch_dgemv<2, PL>(tiling, n, ld, Fh, Fl, D64, xh, xl, U, s); break;
        case 3: launch_dgemv<3, PL>(tiling, n, ld, Fh, Fl, D64, xh, xl, U, s); break;
        default: launch_dgemv<4, PL>(tiling, n, ld, Fh, Fl, D64, xh, xl, U, s); break;
    }
}

// W[d][i] = sum_p Kbar_ip (U[d][j_p] - U[d][i]) = ((Kbar - P) U)_i  (Eq. 16-17), FP64, for
// directions d0 .. d0 + CG - 1.  LPR lanes per row (32 for long sodium rows, 8 for the
// ~50-entry carbon rows): the lanes stride over the row's neighbours (coalesced CSR reads,
// each entry read once for all CG directions), then sum in a fixed butterfly order.
// (Forming the first Gram-Schmidt pass's dots here as well, from the block's rows, measured
// 2x slower than this kernel and k_rdot_part apart: a block holds too few rows for them.)
template <int CG, int LPR>
__global__ void __launch_bounds__(256) k_sparse_real(int64_t n, int d0, const int64_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ col, const double *__restrict__ val,
                                                     const double *__restrict__ U, double *__restrict__ W) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR;
    const int lane = threadIdx.x & (LPR - 1);
    const bool row_ok = i < n;   // rows past n still join the shuffles below
    double ui[CG], acc[CG];
#pragma unroll
    for (int d = 0; d < CG; ++d) {
        ui[d] = row_ok ? U[(int64_t)(d0 + d) * n + i] : 0.0;
        acc[d] = 0.0;
    }
    if (row_ok) {
        const int64_t p0 = rowptr[i], p1 = rowptr[i + 1];
        for (int64_t p = p0 + lane; p < p1; p += LPR) {
            const double v = val[p];
            const int64_t j = col[p];
#pragma unroll
            for (int d = 0; d < CG; ++d) acc[d] += v * (U[(int64_t)(d0 + d) * n + j] - ui[d]);
        }
    }
#pragma unroll
    for (int d = 0; d < CG; ++d) {
#pragma unroll
        for (int off = LPR / 2; off > 0; off >>= 1) acc[d] += __shfl_xor_sync(0xffffffffu, acc[d], off);
    }
    if (row_ok && lane == 0)
#pragma unroll
        for (int d = 0; d < CG; ++d) W[(int64_t)(d0 + d) * n + i] = acc[d];
}

// W[d][i] = R[i * C + d]   (atom-major right-hand sides -> direction-major vectors)
__global__ void k_take_rhs(int64_t n, int C, const double *__restrict__ R, double *__restrict__ W) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * C) return;
    const int64_t d = e / n, i = e - d * n;
    W[e] = R[i * C + d];
}

// ------------------------------------------------------------------ Arnoldi (CGS2, FP64)

constexpr int KV = 8;   // basis vectors per dot-product block

// partial[(rb * nv + k) * C + d] = sum over the rows of block rb of V_k[d][i] w[d][i]
// for k < nv (vectors V + k * vstride), d = blockIdx.z.  Fixed-order reductions.
__global__ void __launch_bounds__(256) k_rdot_part(int64_t n, int C, int nv, const double *__restrict__ V,
                                                   int64_t vstride, const double *__restrict__ w, int64_t rpb,
                                                   double *__restrict__ partial) {
    __shared__ double red[8][KV];
    const int rb = blockIdx.x, d = blockIdx.z, k0 = blockIdx.y * KV;
    const int kn = min(KV, nv - k0);
    const int64_t r0 = (int64_t)rb * rpb, r1 = min(n, r0 + rpb);
    double acc[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) acc[k] = 0.0;
    const double *wd = w + (int64_t)d * n;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += 256) {
        const double wi = wd[i];
#pragma unroll
        for (int k = 0; k < KV; ++k)
            if (k < kn) acc[k] += V[(int64_t)(k0 + k) * vstride + (int64_t)d * n + i] * wi;
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < KV; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[wp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kn) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q) s += red[q][threadIdx.x];
        partial[((int64_t)rb * nv + k0 + threadIdx.x) * C + d] = s;
    }
}

enum { RF_SET = 0, RF_ADD = 1, RF_NORM = 2 };

// One warp per output (k, d): s = sum_rb partial (fixed order).
//   RF_SET : H[d][j][k] = s, coef[k * C + d] = s
//   RF_ADD : H[d][j][k] += s, coef[k * C + d] = s
//   RF_NORM: H[d][j][j + 1] = sqrt(s), hn[d] = sqrt(s)   (nv = 1)
__global__ void k_rdot_fin(int nrb, int nv, int C, int mode, const double *__restrict__ partial, int m, int j,
                           double *__restrict__ H, double *__restrict__ coef, double *__restrict__ hn) {
    const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (o >= (int64_t)nv * C) return;
    const int k = (int)(o / C), d = (int)(o % C);
    double s = 0.0;
    for (int rb = lane; rb < nrb; rb += 32) s += partial[((int64_t)rb * nv + k) * C + d];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane != 0) return;
    if (mode == RF_NORM) {
        const double nr = sqrt(s);
        if (j >= 0) H[((int64_t)d * m + j) * (m + 1) + j + 1] = nr;
        hn[d] = nr;
        return;
    }
    double *hcol = H + ((int64_t)d * m + j) * (m + 1);
    hcol[k] = mode == RF_SET ? s : hcol[k] + s;
    coef[o] = s;
}

constexpr int RU_SLICES = 8;   // warps per block of the Gram-Schmidt updates
constexpr int RU_EPL = 4;      // elements per lane: a block covers RU_ELEMS consecutive rows
constexpr int RU_ELEMS = 32 * RU_EPL;

// w[d][i] -= sum_{k < nv} coef[k * C + d] V_k[d][i] on a grid of (RU_ELEMS-row blocks,
// directions): the block's 8 warps take the vectors k = warp, warp + 8, ... (each lane 4
// rows 32 apart: coalesced 256-byte rows of V_k, two vectors in flight) and their 8 partial
// sums are added in a fixed order.  Fused with the next step's reductions of the updated w:
// NEXT_DOTS -- the partial dots of w with V_0 .. V_{nv-1} for the second Gram-Schmidt pass,
// partial[(block * nv + k) * C + d]; NEXT_NORM -- the partial squared norm,
// partial[block * C + d].  Fixed orders throughout.
enum { NEXT_DOTS = 1, NEXT_NORM = 2 };
template <int NEXT>
__global__ void __launch_bounds__(32 * RU_SLICES) k_rupdate_next(int64_t n, int C, int nv, const double *__restrict__ V,
                                                                 int64_t vstride, const double *__restrict__ coef,
                                                                 double *__restrict__ w, double *__restrict__ partial) {
    __shared__ double part[RU_SLICES][RU_ELEMS];
    __shared__ double wv[RU_ELEMS];
    __shared__ double sqw[RU_ELEMS / 32];
    const int el = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int d = blockIdx.y;
    const int64_t i0 = (int64_t)blockIdx.x * RU_ELEMS;
    const double *Vd = V + (int64_t)d * n + i0;
    double a[RU_EPL];
#pragma unroll
    for (int r = 0; r < RU_EPL; ++r) a[r] = 0.0;
    int k = sl;
    for (; k + RU_SLICES < nv; k += 2 * RU_SLICES) {
        const double c0 = coef[k * C + d], c1 = coef[(k + RU_SLICES) * C + d];
        const double *v0 = Vd + (int64_t)k * vstride, *v1 = v0 + (int64_t)RU_SLICES * vstride;
#pragma unroll
        for (int r = 0; r < RU_EPL; ++r) {
            const int e = el + 32 * r;
            if (i0 + e < n) a[r] += c0 * v0[e] + c1 * v1[e];
        }
    }
    if (k < nv) {
        const double c0 = coef[k * C + d];
        const double *v0 = Vd + (int64_t)k * vstride;
#pragma unroll
        for (int r = 0; r < RU_EPL; ++r) {
            const int e = el + 32 * r;
            if (i0 + e < n) a[r] += c0 * v0[e];
        }
    }
#pragma unroll
    for (int r = 0; r < RU_EPL; ++r) part[sl][el + 32 * r] = a[r];
    __syncthreads();
    if (threadIdx.x < RU_ELEMS) {   // warps 0 .. RU_EPL - 1: one row each
        const int e = threadIdx.x;
        double wn = 0.0;
        if (i0 + e < n) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < RU_SLICES; ++q) t += part[q][e];
            double *we = w + (int64_t)d * n + i0 + e;
            wn = *we - t;
            *we = wn;
        }
        wv[e] = wn;
        if (NEXT == NEXT_NORM) {
            double sq = wn * wn;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
            if (el == 0) sqw[sl] = sq;
        }
    }
    __syncthreads();
    if constexpr (NEXT == NEXT_NORM) {
        if (threadIdx.x == 0) {
            double sq = 0.0;
#pragma unroll
            for (int q = 0; q < RU_ELEMS / 32; ++q) sq += sqw[q];
            partial[(int64_t)blockIdx.x * C + d] = sq;
        }
        return;
    }
    if constexpr (NEXT == NEXT_DOTS)
    for (int k0 = sl; k0 < nv; k0 += 2 * RU_SLICES) {
        double v[2] = {0.0, 0.0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kk = k0 + h * RU_SLICES;
            if (kk >= nv) continue;
            const double *vk = Vd + (int64_t)kk * vstride;
#pragma unroll
            for (int r = 0; r < RU_EPL; ++r) {
                const int e = el + 32 * r;
                if (i0 + e < n) v[h] += vk[e] * wv[e];
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
            v[1] += __shfl_xor_sync(0xffffffffu, v[1], off);
        }
        if (el == 0) {
            partial[((int64_t)blockIdx.x * nv + k0) * C + d] = v[0];
            if (k0 + RU_SLICES < nv) partial[((int64_t)blockIdx.x * nv + k0 + RU_SLICES) * C + d] = v[1];
        }
    }
}

// The norms of the C directions from their nrb partial squares (every block reduces them
// in the same fixed order: lane-strided sums, a butterfly), H(j + 1, j) = hn[d] = norm
// (block 0), then v = w / norm with v's float-pair split, as k_rscale.  Four elements
// per thread.
__global__ void k_rscale_norm(int64_t n, int C, int nrb, const double *__restrict__ partial, int m, int j,
                              double *__restrict__ H, double *__restrict__ hn, const double *__restrict__ w,
                              double *__restrict__ v, float *__restrict__ xh, float *__restrict__ xl) {
    extern __shared__ double nrm[];   // [C]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = warp; d < C; d += blockDim.x / 32) {
        double sv = 0.0;
        for (int rb = lane; rb < nrb; rb += 32) sv += partial[(int64_t)rb * C + d];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
        if (lane == 0) {
            const double nr = sqrt(sv);
            nrm[d] = nr;
            if (blockIdx.x == 0) {
                H[((int64_t)d * m + j) * (m + 1) + j + 1] = nr;
                hn[d] = nr;
            }
        }
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        const int64_t e = ((int64_t)blockIdx.x * 4 + q) * blockDim.x + threadIdx.x;
        if (e >= n * C) break;
        const double h = nrm[e / n];
        const double t = h > 0.0 ? w[e] / h : 0.0;
        v[e] = t;
        df_split(t, xh[e], xl[e]);
    }
}

// v[d][i] = w[d][i] / hn[d] (0 when hn = 0: the direction's Krylov space is exhausted),
// and v's float-pair split (xh, xl) for the next D product
__global__ void k_rscale(int64_t n, int C, const double *__restrict__ hn, const double *__restrict__ w,
                         double *__restrict__ v, float *__restrict__ xh, float *__restrict__ xl) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * C) return;
    const double h = hn[e / n];
    const double t = h > 0.0 ? w[e] / h : 0.0;
    v[e] = t;
    df_split(t, xh[e], xl[e]);
}

// ------------------------------------------------------------------ per-shift least squares

struct ShiftDev {
    int m;
    int64_t ncols;
    int C;
    const double *H;     // [C][m][m + 1]: column j of direction d at (d * m + j) * (m + 1)
    const int *cdir;     // [ncols] direction of each column
    const double2 *z;    // [ncols] shift z(omega_c)
    double *cs;          // [m][ncols]
    double2 *sn;         // [m][ncols]
    double2 *g;          // [m + 1][ncols]
    double2 *Rt;         // [m (m + 1) / 2][ncols] rotated Hbar - z Ibar, column j at j (j + 1) / 2
    const double *target;  // [C] residual-estimate target per direction
    int *done;           // [ncols]
    int *jdone;          // [ncols] Arnoldi steps the column uses
};

// g0 = ||R_d|| e1 for every column
__global__ void k_shift_init(ShiftDev st, const double *__restrict__ rn) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st.ncols) return;
    const double r = rn[st.cdir[c]];
    st.g[c] = make_double2(r, 0.0);
    st.done[c] = r == 0.0 ? 1 : 0;
    st.jdone[c] = 0;
}

// Column j of Hbar - z Ibar for one column: apply the previous rotations, form the new one
// (complex sine, real cosine), update g; done when |g_{j+1}| <= target or the process
// broke down (H(j+1, j) = 0: the Krylov space is invariant, the iterate exact).
// h: entries 0..j of column j of the column's direction; hb = H(j+1, j).
__device__ void shift_givens_col(const ShiftDev &st, int64_t c, int j, const double *h, double hb) {
    if (st.done[c]) return;
    const int64_t nc = st.ncols;
    const int d = st.cdir[c];
    const double *__restrict__ csv = st.cs + c;
    const double2 *__restrict__ snv = st.sn + c;
    const double2 zc = st.z[c];
    double2 *__restrict__ R = st.Rt + (int64_t)j * (j + 1) / 2 * nc + c;
    // t_i = h_i - z delta_ij, rotated by G_0 .. G_{j-1}.  The rotations' loads do not depend
    // on the chain, so they are issued eight at a time ahead of it.
    double2 prev = make_double2(h[0] - (j == 0 ? zc.x : 0.0), j == 0 ? -zc.y : 0.0);
    int i = 0;
    for (; i + 8 <= j; i += 8) {
        double csr[8], hr[8];
        double2 snr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            csr[u] = __ldg(csv + (int64_t)(i + u) * nc);
            snr[u] = __ldg(snv + (int64_t)(i + u) * nc);
            hr[u] = h[i + u + 1];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool diag = i + u + 1 == j;
            const double2 nxt = make_double2(hr[u] - (diag ? zc.x : 0.0), diag ? -zc.y : 0.0);
            R[(int64_t)(i + u) * nc] = c_add(c_scale(csr[u], prev), c_mul(snr[u], nxt));
            prev = c_sub(c_scale(csr[u], nxt), c_conjmul(snr[u], prev));
        }
    }
    for (; i < j; ++i) {
        const double2 nxt = make_double2(h[i + 1] - (i + 1 == j ? zc.x : 0.0), i + 1 == j ? -zc.y : 0.0);
        const double cs = __ldg(csv + (int64_t)i * nc);
        const double2 sn = __ldg(snv + (int64_t)i * nc);
        R[(int64_t)i * nc] = c_add(c_scale(cs, prev), c_mul(sn, nxt));
        prev = c_sub(c_scale(cs, nxt), c_conjmul(sn, prev));
    }
    const double na = sqrt(c_abs2(prev));
    const double nu = sqrt(na * na + hb * hb);
    double cs;
    double2 sn, rdiag;
    if (nu == 0.0) {
        cs = 1.0;
        sn = make_double2(0.0, 0.0);
        rdiag = prev;
    } else if (na == 0.0) {
        cs = 0.0;
        sn = make_double2(1.0, 0.0);
        rdiag = make_double2(hb, 0.0);
    } else {
        const double2 ph = c_scale(1.0 / na, prev);
        cs = na / nu;
        sn = c_scale(hb / nu, ph);
        rdiag = c_scale(nu, ph);
    }
    st.cs[(int64_t)j * nc + c] = cs;
    st.sn[(int64_t)j * nc + c] = sn;
    R[(int64_t)j * nc] = rdiag;
    const double2 gj = st.g[(int64_t)j * nc + c];
    const double2 g1 = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));   // -conj(sn) g_j
    st.g[(int64_t)(j + 1) * nc + c] = g1;
    st.g[(int64_t)j * nc + c] = c_scale(cs, gj);
    if (sqrt(c_abs2(g1)) <= st.target[d] || hb == 0.0 || nu == 0.0) {
        st.done[c] = 1;
        st.jdone[c] = j + 1;
    }
}

__global__ void k_shift_givens(ShiftDev st, int j) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st.ncols) return;
    const double *h = st.H + ((int64_t)st.cdir[c] * st.m + j) * (st.m + 1);
    shift_givens_col(st, c, j, h, h[j + 1]);
}

// y = R^{-1} g over the column's jdone steps (columns still open use jlast + 1), a warp per
// column, column-oriented: for k = jd-1 .. 0, y_k = y_k / R_kk, then y_l -= R_lk y_k for
// l < k.  Column k of R is contiguous in the packed layout; lane l mod 32 owns y_l, and
// the owner of y_k broadcasts it.
__global__ void k_shift_backsolve(ShiftDev st, int jlast, double2 *__restrict__ y) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= st.ncols) return;   // whole warp
    const int64_t nc = st.ncols;
    const int jd = st.done[c] ? st.jdone[c] : jlast + 1;
    const double2 *__restrict__ Rt = st.Rt + c;
    double2 *__restrict__ yc = y + c;
    for (int l = lane; l < jd; l += 32) yc[(int64_t)l * nc] = st.g[(int64_t)l * nc + c];
    for (int k = jd - 1; k >= 0; --k) {
        const int owner = k & 31;
        double2 yk = make_double2(0.0, 0.0);
        if (lane == owner) {
            yk = c_div(yc[(int64_t)k * nc], Rt[((int64_t)k * (k + 1) / 2 + k) * nc]);
            yc[(int64_t)k * nc] = yk;
        }
        yk.x = __shfl_sync(0xffffffffu, yk.x, owner);
        yk.y = __shfl_sync(0xffffffffu, yk.y, owner);
        const int64_t col0 = (int64_t)k * (k + 1) / 2;
        for (int l = lane; l < k; l += 32)
            yc[(int64_t)l * nc] = c_sub(yc[(int64_t)l * nc], c_mul(Rt[(col0 + l) * nc], yk));
    }
    __syncwarp();
    if (lane == 0) st.jdone[c] = jd;
}

// q[i][c] = sum_{k < jdone_c} V_k[d_c][i] y[k][c]
__global__ void k_shift_combine(int64_t n, int64_t nc, const double *__restrict__ V, int64_t vstride,
                                const double2 *__restrict__ y, const int *__restrict__ jdone,
                                const int *__restrict__ cdir, double2 *__restrict__ q) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nc) return;
    const int64_t i = e / nc, c = e - i * nc;
    const double *v = V + (int64_t)cdir[c] * n + i;
    const int jd = jdone[c];
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    int k = 0;
    for (; k + 1 < jd; k += 2) {
        const double v0 = v[(int64_t)k * vstride], v1 = v[(int64_t)(k + 1) * vstride];
        const double2 y0 = y[(int64_t)k * nc + c], y1 = y[(int64_t)(k + 1) * nc + c];
        a.x += v0 * y0.x;
        a.y += v0 * y0.y;
        b.x += v1 * y1.x;
        b.y += v1 * y1.y;
    }
    if (k < jd) {
        const double v0 = v[(int64_t)k * vstride];
        const double2 y0 = y[(int64_t)k * nc + c];
        a.x += v0 * y0.x;
        a.y += v0 * y0.y;
    }
    q[e] = c_add(a, b);
}

__global__ void k_shift_z(int64_t nc, const double *__restrict__ col_omega, ShiftModel zm,
                          double2 *__restrict__ z) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    z[c] = z_eval(zm, col_omega[c]);   // Eq. 12 (omega-FQ) or -Lambda(w) of Eq. 21 (BEM)
}

// ------------------------------------------------------------------ host

struct Arnoldi {
    wfq_geom *g;
    cudaStream_t s;
    int64_t n;
    int C;
    int64_t rpb;
    int nrb;
    DevBuf<float> xh, xl;
    DevBuf<double> U, partial, coef;
    DevBuf<double> partial_f;   // partial reductions of the fused kernels (update + dots / norm)
    int nbru = 0;
    DevBuf<float2> rowpart, colpart;   // symmetric product partial sums

    int init(wfq_geom *geom, int ndir, int m, cudaStream_t stream) {
        g = geom;
        s = stream;
        n = g->n;
        C = ndir;
        rpb = std::max<int64_t>(1024, round_up((n + 2 * g->ctx->num_sms - 1) / (2 * g->ctx->num_sms), 256));
        nrb = (int)((n + rpb - 1) / rpb);
        WFQ_TRY(xh.alloc(g->ctx, (size_t)n * C, s));
        WFQ_TRY(xl.alloc(g->ctx, (size_t)n * C, s));
        WFQ_TRY(U.alloc(g->ctx, (size_t)n * C, s));
        WFQ_TRY(partial.alloc(g->ctx, (size_t)nrb * (m + 1) * C, s));
        nbru = (int)((n + RU_ELEMS - 1) / RU_ELEMS);
        WFQ_TRY(partial_f.alloc(g->ctx, (size_t)nbru * (m + 1) * C, s));
        WFQ_TRY(coef.alloc(g->ctx, (size_t)(m + 1) * C, s));
        if (g->Dsym && !g->Dfh) {
            const int64_t T = g->sym_nt, cg = std::min<int64_t>(C, 4);
            WFQ_TRY(rowpart.alloc(g->ctx, (size_t)g->sym_nitems * kSymTile * cg, s));
            WFQ_TRY(colpart.alloc(g->ctx, (size_t)(T * (T + 1) / 2) * kSymTile * cg, s));
        }
        return WFQ_OK;
    }

    // Tiling of the GEMV for `cg` vectors on this geometry's shape: looked up in the
    // context's autotuner cache, else chosen now by timing every tiling twice on the real
    // operands (xh / xl already split) and kept for later products of the same shape.
    int tiling_for(int cg, bool pl, const float *ph, const float *pl_x, double *pu) {
        const int64_t key = ((int64_t)n << 8) | ((int64_t)cg << 1) | (pl ? 1 : 0);
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
        for (int t = 0; t < GV_NTILINGS; ++t) {
            float ms = 0.f;
            for (int rep = 0; rep < 3; ++rep) {   // the first of the three warms up
                if (rep == 1) cudaEventRecord(e0, s);
                if (pl) launch_dgemv_c<true>(cg, t, n, g->ldf, g->Dfh, g->Dfl, nullptr, ph, pl_x, pu, s);
                else launch_dgemv_c<false>(cg, t, n, n, nullptr, nullptr, g->D64, ph, pl_x, pu, s);
                note_launch();
            }
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lk(g->ctx->tune_mu);
        g->ctx->tuned[key] = best;
        return best;
    }

    // u = D v; xh / xl already hold v's float-pair split (written when v was normalised)
    int dmul(double *u) {
        if (!g->Dsym && !g->Dfh && !g->D64) {   // matrix-free: D regenerated per product
            KScope ks(g->ctx, WFQ_KT_DGEMV_DF, s, 0.0);
            for (int d0 = 0; d0 < C; d0 += 4)
                WFQ_TRY(d_gemv_df_mf(g, std::min(4, C - d0), xh.ptr + (int64_t)d0 * n, xl.ptr + (int64_t)d0 * n,
                                     u + (int64_t)d0 * n, s));
            return WFQ_OK;
        }
        if (g->Dsym && !g->Dfh) {   // symmetric tiles: half the bytes, each tile used twice (the
                                    // full planes, when also stored, measured slightly faster)
            const int64_t T = g->sym_nt;
            const double dbytes = (double)(T * (T + 1) / 2) * 2.0 * kSymTile * kSymTile * 4.0;
            for (int d0 = 0; d0 < C; d0 += 4) {
                const int cg = std::min(4, C - d0);
                const float *ph = xh.ptr + (int64_t)d0 * n, *pxl = xl.ptr + (int64_t)d0 * n;
                KScope ks(g->ctx, WFQ_KT_DGEMV_DF, s, dbytes);
                const unsigned items = (unsigned)g->sym_nitems;
                switch (cg) {
                    case 1: k_dsymv_df<1><<<items, 256, 0, s>>>(n, T, g->Dsym, g->sym_items, ph, pxl, rowpart.ptr, colpart.ptr); break;
                    case 2: k_dsymv_df<2><<<items, 256, 0, s>>>(n, T, g->Dsym, g->sym_items, ph, pxl, rowpart.ptr, colpart.ptr); break;
                    case 3: k_dsymv_df<3><<<items, 256, 0, s>>>(n, T, g->Dsym, g->sym_items, ph, pxl, rowpart.ptr, colpart.ptr); break;
                    default: k_dsymv_df<4><<<items, 256, 0, s>>>(n, T, g->Dsym, g->sym_items, ph, pxl, rowpart.ptr, colpart.ptr); break;
                }
                note_launch();
                k_dsymv_finish<<<nblk(n * cg), 256, 0, s>>>(n, cg, T, g->sym_item_start, rowpart.ptr, colpart.ptr,
                                                           u + (int64_t)d0 * n);
                note_launch();
            }
            WFQ_CUDA(cudaGetLastError());
            return WFQ_OK;
        }
        const double dbytes = 8.0 * (double)n * (double)n;   // algorithmic: the N^2 entries, 8 bytes each
        const bool pl = g->Dfh != nullptr;
        for (int d0 = 0; d0 < C; d0 += 4) {
            const int cg = std::min(4, C - d0);
            const float *ph = xh.ptr + (int64_t)d0 * n, *pxl = xl.ptr + (int64_t)d0 * n;
            double *pu = u + (int64_t)d0 * n;
            const int tiling = tiling_for(cg, pl, ph, pxl, pu);
            KScope ks(g->ctx, WFQ_KT_DGEMV_DF, s, dbytes);
            if (pl) launch_dgemv_c<true>(cg, tiling, n, g->ldf, g->Dfh, g->Dfl, nullptr, ph, pxl, pu, s);
            else launch_dgemv_c<false>(cg, tiling, n, n, nullptr, nullptr, g->D64, ph, pxl, pu, s);
            note_launch();
        }
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }

    // lanes per row of the sparse term: a full warp for long (sodium) rows, 8 for carbon rows
    int sparse_lpr() const { return g->nnz > 128 * n ? 32 : 8; }

    // w = (Kbar - P) u; BEM geometries (A = the stored operator itself): w = u
    int sparse(const double *u, double *w) {
        KScope ks(g->ctx, WFQ_KT_SPARSE, s);
        if (g->op == OP_BEM) {
            WFQ_CUDA(cudaMemcpyAsync(w, u, sizeof(double) * n * C, cudaMemcpyDeviceToDevice, s));
            return WFQ_OK;
        }
        const bool wide = sparse_lpr() == 32;
        const unsigned blocks = nblk(n * (wide ? 32 : 8));
        for (int d0 = 0; d0 < C; d0 += 4) {
            const int cg = std::min(4, C - d0);
#define WFQ_SP(CC)                                                                                    \
    if (wide)                                                                                         \
        k_sparse_real<CC, 32><<<blocks, 256, 0, s>>>(n, d0, g->rowptr, g->col, g->val64, u, w);      \
    else                                                                                              \
        k_sparse_real<CC, 8><<<blocks, 256, 0, s>>>(n, d0, g->rowptr, g->col, g->val64, u, w);
            switch (cg) {
                case 1: WFQ_SP(1) break;
                case 2: WFQ_SP(2) break;
                case 3: WFQ_SP(3) break;
                default: WFQ_SP(4) break;
            }
#undef WFQ_SP
            note_launch();
        }
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }

    // dots of w with nv vectors V_0.. (stride vstride), finished into H column j / coef / hn
    int dots(const double *V, int64_t vstride, int nv, const double *w, int mode, int m, int j, double *H, double *hn) {
        dim3 grid((unsigned)nrb, (unsigned)((nv + KV - 1) / KV), (unsigned)C);
        k_rdot_part<<<grid, 256, 0, s>>>(n, C, nv, V, vstride, w, rpb, partial.ptr); note_launch();
        k_rdot_fin<<<nblk((int64_t)nv * C * 32), 256, 0, s>>>(nrb, nv, C, mode, partial.ptr, m, j, H, coef.ptr, hn); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }
};

// Real column r of an atom-major complex block X (n x cc; r = 2c + 0/1 for the real and
// imaginary parts of column c) split into direction-major float pairs xh/xl [C][n].
__global__ void k_cols_split(int64_t n, int C, const double *__restrict__ X, float *__restrict__ xh,
                             float *__restrict__ xl) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * C) return;
    const int64_t r = e / n, i = e - r * n;
    df_split(X[i * C + r], xh[e], xl[e]);
}

// U (atom-major complex block, real column r at i * C + r) = Ud [C][n]
__global__ void k_cols_gather(int64_t n, int C, const double *__restrict__ Ud, double *__restrict__ U) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * C) return;
    const int64_t i = e / C, r = e - i * C;
    U[e] = Ud[r * n + i];
}

}  // namespace

int d_apply_pairs_df(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s) {
    const int64_t n = g->n;
    const int C = (int)(2 * cc);
    if (!(g->Dfh || g->Dsym)) return fail(WFQ_EUNSUPPORTED, "float-pair product: needs stored pairs");
    DevBuf<float> xh, xl;
    DevBuf<double> ud, rowpart, colpart;
    WFQ_TRY(xh.alloc(g->ctx, (size_t)n * C, s));
    WFQ_TRY(xl.alloc(g->ctx, (size_t)n * C, s));
    WFQ_TRY(ud.alloc(g->ctx, (size_t)n * C, s));
    k_cols_split<<<nblk(n * C), 256, 0, s>>>(n, C, reinterpret_cast<const double *>(X), xh.ptr, xl.ptr);
    note_launch();
    KScope ks(g->ctx, WFQ_KT_DAPPLY_FP64, s, 2.0 * (double)n * (double)n * (double)C);
    if (g->Dfh) {
        for (int d0 = 0; d0 < C; d0 += 4) {
            const int cg = std::min(4, C - d0);
            launch_dgemv_c<true>(cg, 0, n, g->ldf, g->Dfh, g->Dfl, nullptr, xh.ptr + (int64_t)d0 * n,
                                 xl.ptr + (int64_t)d0 * n, ud.ptr + (int64_t)d0 * n, s);
            note_launch();
        }
    } else {
        const int64_t T = g->sym_nt;
        WFQ_TRY(rowpart.alloc(g->ctx, (size_t)g->sym_nitems * kSymTile * 4 * 2, s));
        WFQ_TRY(colpart.alloc(g->ctx, (size_t)(T * (T + 1) / 2) * kSymTile * 4 * 2, s));
        float2 *rp = reinterpret_cast<float2 *>(rowpart.ptr), *cp = reinterpret_cast<float2 *>(colpart.ptr);
        for (int d0 = 0; d0 < C; d0 += 4) {
            const int cg = std::min(4, C - d0);
            const float *ph = xh.ptr + (int64_t)d0 * n, *pxl = xl.ptr + (int64_t)d0 * n;
            const unsigned items = (unsigned)g->sym_nitems;
            switch (cg) {
                case 1: k_dsymv_df<1><<<items, 256, 0, s>>>(n, T, g->Dsym, g->sym_items, ph, pxl, rp, cp); break;
                case 2: k_dsymv_df<2><<<items, 256, 0, s>>>(n, T, g->Dsym, g->sym_items, ph, pxl, rp, cp); break;
                case 3: k_dsymv_df<3><<<items, 256, 0, s>>>(n, T, g->Dsym, g->sym_items, ph, pxl, rp, cp); break;
                default: k_dsymv_df<4><<<items, 256, 0, s>>>(n, T, g->Dsym, g->sym_items, ph, pxl, rp, cp); break;
            }
            note_launch();
            k_dsymv_finish<<<nblk(n * cg), 256, 0, s>>>(n, cg, T, g->sym_item_start, rp, cp, ud.ptr + (int64_t)d0 * n);
            note_launch();
        }
    }
    k_cols_gather<<<nblk(n * C), 256, 0, s>>>(n, C, ud.ptr, reinterpret_cast<double *>(U));
    note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

int d_apply_mf_gemv_df(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s) {
    const int64_t n = g->n;
    const int C = (int)(2 * cc);
    if (C > 8) return fail(WFQ_EUNSUPPORTED, "matrix-free double-float GEMV: at most 4 complex columns");
    DevBuf<float> xh, xl;
    DevBuf<double> ud;
    WFQ_TRY(xh.alloc(g->ctx, (size_t)n * C, s));
    WFQ_TRY(xl.alloc(g->ctx, (size_t)n * C, s));
    WFQ_TRY(ud.alloc(g->ctx, (size_t)n * C, s));
    k_cols_split<<<nblk(n * C), 256, 0, s>>>(n, C, reinterpret_cast<const double *>(X), xh.ptr, xl.ptr);
    note_launch();
    KScope ks(g->ctx, WFQ_KT_DAPPLY_FP64, s, 2.0 * (double)n * (double)n * (double)C);
    for (int d0 = 0; d0 < C; d0 += 4)
        WFQ_TRY(d_gemv_df_mf(g, std::min(4, C - d0), xh.ptr + (int64_t)d0 * n, xl.ptr + (int64_t)d0 * n,
                             ud.ptr + (int64_t)d0 * n, s));
    k_cols_gather<<<nblk(n * C), 256, 0, s>>>(n, C, ud.ptr, reinterpret_cast<double *>(U));
    note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

size_t shifted_footprint(const wfq_geom *g, int64_t ncols, int ndir, int m) {
    if (m <= 0) m = 600;
    const size_t n = (size_t)g->n, C = (size_t)ndir, nc = (size_t)ncols;
    size_t b = (size_t)(2 * m + 1) * n * C * 8;                                // Arnoldi vectors, D v_k
    b += (size_t)m * (m + 1) / 2 * nc * 16 + (size_t)(3 * m + 2) * nc * 16;   // rotated H, rotations, g, y
    b += n * nc * 16 * 9;                                                     // q, D q, residual blocks
    return b;
}

int solve_gmres_shifted(wfq_geom *g, const SolveArgs &a, cudaStream_t s) {
    wfq_ctx *ctx = g->ctx;
    const int64_t n = g->n, C = a.ndir, nc = a.col_omega ? a.ncols : a.nfreq * C;
    int m = a.m > 0 ? a.m : 600;
    m = std::max(1, std::min(m, a.max_iter));
    if ((double)n * C * (2 * m + 1) * 8.0 > 0.5 * 284e9)
        return fail(WFQ_ENOMEM, "shifted GMRES basis (Arnoldi vectors and their D products) does not fit: lower m");

    Arnoldi ar;
    WFQ_TRY(ar.init(g, (int)C, m, s));
    const int64_t vstride = n * C;
    DevBuf<double> V, DV, H, hn, R, dirs, om, cs, target;
    DevBuf<double2> z, sn, gv, Rt, y, dq;
    DevBuf<int> cdir, done, jdone;
    WFQ_TRY(V.alloc(ctx, (size_t)(m + 1) * vstride, s));
    WFQ_TRY(DV.alloc(ctx, (size_t)m * vstride, s));   // D v_k of every Arnoldi vector used
    WFQ_TRY(H.alloc(ctx, (size_t)C * m * (m + 1), s));
    WFQ_TRY(hn.alloc(ctx, C, s));
    WFQ_TRY(R.alloc(ctx, (size_t)n * C, s));
    WFQ_TRY(dirs.alloc(ctx, 3 * C, s));
    WFQ_TRY(om.alloc(ctx, nc, s));
    WFQ_TRY(cs.alloc(ctx, (size_t)m * nc, s));
    WFQ_TRY(target.alloc(ctx, C, s));
    WFQ_TRY(z.alloc(ctx, nc, s));
    WFQ_TRY(sn.alloc(ctx, (size_t)m * nc, s));
    WFQ_TRY(gv.alloc(ctx, (size_t)(m + 1) * nc, s));
    WFQ_TRY(Rt.alloc(ctx, (size_t)m * (m + 1) / 2 * nc, s));
    WFQ_TRY(y.alloc(ctx, (size_t)m * nc, s));
    WFQ_TRY(cdir.alloc(ctx, nc, s));
    WFQ_TRY(done.alloc(ctx, nc, s));
    WFQ_TRY(jdone.alloc(ctx, nc, s));
    // column c: frequency om_h[c], direction cdir_h[c] (explicit lists, or c = f * ndir + d)
    std::vector<int> cdir_h(nc);
    std::vector<double> om_h(nc);
    for (int64_t c = 0; c < nc; ++c) {
        cdir_h[c] = a.col_dir ? a.col_dir[c] : (int)(c % C);
        om_h[c] = a.col_omega ? a.col_omega[c] : a.omega[c / C];
    }
    WFQ_CUDA(cudaMemcpyAsync(cdir.ptr, cdir_h.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    WFQ_CUDA(cudaMemcpyAsync(dirs.ptr, a.dirs, sizeof(double) * 3 * C, cudaMemcpyHostToDevice, s));
    WFQ_CUDA(cudaMemcpyAsync(om.ptr, om_h.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, s));
    WFQ_CUDA(cudaMemsetAsync(H.ptr, 0, sizeof(double) * C * m * (m + 1), s));
    k_shift_z<<<nblk(nc), 256, 0, s>>>(nc, om.ptr, shift_model(g), z.ptr); note_launch();

    // v_0 = R_d / ||R_d||
    WFQ_TRY(launch_rhs(g, (int)C, dirs.ptr, a.E0, R.ptr, s));
    k_take_rhs<<<nblk(n * C), 256, 0, s>>>(n, (int)C, R.ptr, ar.U.ptr); note_launch();
    WFQ_TRY(ar.dots(ar.U.ptr, 0, 1, ar.U.ptr, RF_NORM, m, -1, H.ptr, hn.ptr));
    k_rscale<<<nblk(n * C), 256, 0, s>>>(n, (int)C, hn.ptr, ar.U.ptr, V.ptr, ar.xh.ptr, ar.xl.ptr); note_launch();
    std::vector<double> rn_h(C), tg(C);
    WFQ_CUDA(cudaMemcpyAsync(rn_h.data(), hn.ptr, sizeof(double) * C, cudaMemcpyDeviceToHost, s));
    WFQ_CUDA(cudaStreamSynchronize(s));   // also completes the cdir_h / om_h uploads
    for (int64_t d = 0; d < C; ++d) tg[d] = 0.5 * a.rel_tol * rn_h[d];
    WFQ_CUDA(cudaMemcpyAsync(target.ptr, tg.data(), sizeof(double) * C, cudaMemcpyHostToDevice, s));
    ShiftDev st{m, nc, (int)C, H.ptr, cdir.ptr, z.ptr, cs.ptr, sn.ptr, gv.ptr, Rt.ptr, target.ptr, done.ptr, jdone.ptr};
    k_shift_init<<<nblk(nc), 256, 0, s>>>(st, hn.ptr); note_launch();
    WFQ_CUDA(cudaGetLastError());

    std::vector<int> done_h(nc);
    int jlast = -1;
    // The per-frequency Givens step of iteration j needs only column j of H, so it runs on a
    // side stream, overlapped with the next iteration's D product; the solve stream joins it
    // before every convergence check and before the back substitution.
    struct SideStream {
        cudaStream_t st = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
        ~SideStream() {
            if (st) {
                cudaStreamSynchronize(st);
                cudaStreamDestroy(st);
            }
            if (fork) cudaEventDestroy(fork);
            if (join) cudaEventDestroy(join);
        }
    } side;
    WFQ_CUDA(cudaStreamCreateWithFlags(&side.st, cudaStreamNonBlocking));
    WFQ_CUDA(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming));
    WFQ_CUDA(cudaEventCreateWithFlags(&side.join, cudaEventDisableTiming));
    auto join_side = [&]() -> int {
        WFQ_CUDA(cudaEventRecord(side.join, side.st));
        WFQ_CUDA(cudaStreamWaitEvent(s, side.join, 0));
        return WFQ_OK;
    };
    for (int j = 0; j < m; ++j) {
        double *dvj = DV.ptr + (int64_t)j * vstride;
        double *w = V.ptr + (int64_t)(j + 1) * vstride;
        WFQ_TRY(ar.dmul(dvj));
        // w = (Kbar - P) D v_j, the first classical Gram-Schmidt pass's dots; each update of
        // the two passes forms the partial reductions of the next step (the second pass's
        // dots, then the norm): 9 launches per step with the D product and the Givens step
        // (12 with a launch per reduction).  Finishing the first pass's dots inside the first
        // update as well (8 launches) measured slower: 102.3-102.7 against 101.1 ms per
        // cnt20k step, the finish then a serial prologue of every update block.
        WFQ_TRY(ar.sparse(dvj, w));
        {
            KScope ko(ctx, WFQ_KT_ORTHO, s);
            const int nv = j + 1;
            WFQ_TRY(ar.dots(V.ptr, vstride, nv, w, RF_SET, m, j, H.ptr, hn.ptr));
            k_rupdate_next<NEXT_DOTS><<<dim3((unsigned)ar.nbru, (unsigned)C), 32 * RU_SLICES, 0, s>>>(
                n, (int)C, nv, V.ptr, vstride, ar.coef.ptr, w, ar.partial_f.ptr);
            note_launch();
            k_rdot_fin<<<nblk((int64_t)nv * C * 32), 256, 0, s>>>(ar.nbru, nv, (int)C, RF_ADD, ar.partial_f.ptr, m, j,
                                                                  H.ptr, ar.coef.ptr, hn.ptr);
            note_launch();
            k_rupdate_next<NEXT_NORM><<<dim3((unsigned)ar.nbru, (unsigned)C), 32 * RU_SLICES, 0, s>>>(
                n, (int)C, nv, V.ptr, vstride, ar.coef.ptr, w, ar.partial_f.ptr);
            note_launch();
            k_rscale_norm<<<nblk(n * C, 1024), 256, sizeof(double) * C, s>>>(n, (int)C, ar.nbru, ar.partial_f.ptr, m,
                                                                             j, H.ptr, hn.ptr, w, w, ar.xh.ptr,
                                                                             ar.xl.ptr);
            note_launch();
            WFQ_CUDA(cudaEventRecord(side.fork, s));
            WFQ_CUDA(cudaStreamWaitEvent(side.st, side.fork, 0));
            k_shift_givens<<<nblk(nc, PER_COLUMN_BLOCK), PER_COLUMN_BLOCK, 0, side.st>>>(st, j); note_launch();
            WFQ_CUDA(cudaGetLastError());
        }
        jlast = j;
        if ((j & 3) == 3 || j == m - 1) {
            WFQ_TRY(join_side());
            WFQ_CUDA(cudaMemcpyAsync(done_h.data(), done.ptr, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
            WFQ_TRY(check_device_error(ctx, s));
            if (std::all_of(done_h.begin(), done_h.end(), [](int v) { return v != 0; })) break;
        }
    }
    WFQ_TRY(join_side());
    WFQ_TRY(dq.alloc(ctx, (size_t)n * nc, s));
    k_shift_backsolve<<<nblk(nc * 32, 128), 128, 0, s>>>(st, jlast, y.ptr); note_launch();
    k_shift_combine<<<nblk(n * nc), 256, 0, s>>>(n, nc, V.ptr, vstride, y.ptr, jdone.ptr, cdir.ptr, a.q); note_launch();
    k_shift_combine<<<nblk(n * nc), 256, 0, s>>>(n, nc, DV.ptr, vstride, y.ptr, jdone.ptr, cdir.ptr, dq.ptr); note_launch();
    WFQ_CUDA(cudaGetLastError());
    std::vector<int> jd_h(nc);
    WFQ_CUDA(cudaMemcpyAsync(jd_h.data(), jdone.ptr, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
    WFQ_CUDA(cudaStreamSynchronize(s));

    trace("shifted gmres: %d Arnoldi steps for %lld columns (%lld directions)", jlast + 1, (long long)nc,
          (long long)C);
    // FP64 true residual of every column; the ones above tol continue in block GMRES(50)
    return finish_columns(g, a, jd_h, 50, dq.ptr, s);
}

}  // namespace wfq
