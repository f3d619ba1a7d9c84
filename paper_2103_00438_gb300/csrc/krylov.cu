// Krylov shells of Section 3 on the GPU, batched over independent complex columns
// (one column per (frequency, field direction); all columns share D and Kbar).
//
//   GMRES / GMRES(m) (Eq. 24): Arnoldi with iterated classical Gram-Schmidt (two
//     projection passes, "CGS2"), Givens QR of the Hessenberg matrix, x = x0 + V y.
//     Inner products, norms, rotations and the solution update are FP64; the basis is
//     complex128 (FP64 operator) or complex64 (mixed operator).  Every restart cycle
//     starts from the FP64 true residual r = R - (A - zI) x (iterative refinement of the
//     mixed form), and only the columns that have not converged take part in it: the
//     block is compacted at every cycle boundary.
//   J-symmetric QMR from BCG without look-ahead (J = D, Eq. 18): BCG with shadow vectors
//     J r and J p smoothed into the QMR iterate.  D p for A p comes from the recurrence
//     D p <- D r + beta D p, so one D product (D r) per iteration serves both A p and the
//     bilinear form r^T D r.
//
// Column reductions are deterministic two-stage sums: per-block partials over a fixed
// split of the atom rows, then one warp per output summing the partials in block order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"

namespace wfq {

// FP64-grade product of the FP64 solvers' Arnoldi and QMR iterations (their true residuals
// take d_apply_fp64). With no FP64 D stored, the double-float product (~2^-48 per product,
// on the FP32 pipes: the stored float-pair planes or tiles, else D regenerated per product)
// instead of D regenerated in FP64: on GB300's FP64 rate the latter is ~8 s per 192-column
// product at 1.5e5 atoms and ~100 s per 32-column product at 10^6 atoms, the double-float
// forms 4 to 6 times less.
static int solver_fp64_product(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s) {
    if (!g->D64 && g->op == OP_WFQ) return d_apply_df(g, cc, X, U, s);
    return d_apply_fp64(g, cc, X, U, s);
}

// ------------------------------------------------------------------ complex helpers

__device__ __forceinline__ double2 ld2(const double2 *p) { return *p; }
__device__ __forceinline__ double2 ld2(const float2 *p) {
    float2 v = *p;
    return make_double2(v.x, v.y);
}
__device__ __forceinline__ void st2(double2 *p, double2 v) { *p = v; }
__device__ __forceinline__ void st2(float2 *p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cjmul(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 czero() { return make_double2(0.0, 0.0); }

static inline unsigned nblocks(int64_t total, int t = 256) { return (unsigned)((total + t - 1) / t); }

// ------------------------------------------------------------------ per-thread accumulators
// FP64 vectors accumulate in FP64.  complex64 vectors accumulate in double-float: each
// real product is split exactly into p + e (FMA) and added with Knuth's two-sum, so the
// running sum keeps ~48 bits on the FP32 pipes (GB300's FP64 rate is far lower).

__device__ __forceinline__ void df_fma(float a, float b, float &h, float &l) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const float s = __fadd_rn(h, p);
    const float v = __fsub_rn(s, h);
    const float t = __fadd_rn(__fsub_rn(h, __fsub_rn(s, v)), __fsub_rn(p, v));
    h = s;
    l += t + e;
}

template <class VT>
struct Acc;

template <>
struct Acc<double2> {
    double2 v;
    __device__ __forceinline__ void zero() { v = make_double2(0.0, 0.0); }
    __device__ __forceinline__ void cdot(double2 a, double2 w) {  // += conj(a) w
        v.x += a.x * w.x + a.y * w.y;
        v.y += a.x * w.y - a.y * w.x;
    }
    __device__ __forceinline__ void bilin(double2 a, double2 w) {  // += a w
        v.x += a.x * w.x - a.y * w.y;
        v.y += a.x * w.y + a.y * w.x;
    }
    __device__ __forceinline__ void norm2(double2 w) { v.x += w.x * w.x + w.y * w.y; }
    __device__ __forceinline__ double2 get() const { return v; }
};

template <>
struct Acc<float2> {
    float rh, rl, ih, il;
    __device__ __forceinline__ void zero() { rh = rl = ih = il = 0.f; }
    __device__ __forceinline__ void cdot(float2 a, float2 w) {
        df_fma(a.x, w.x, rh, rl);
        df_fma(a.y, w.y, rh, rl);
        df_fma(a.x, w.y, ih, il);
        df_fma(-a.y, w.x, ih, il);
    }
    __device__ __forceinline__ void bilin(float2 a, float2 w) {
        df_fma(a.x, w.x, rh, rl);
        df_fma(-a.y, w.y, rh, rl);
        df_fma(a.x, w.y, ih, il);
        df_fma(a.y, w.x, ih, il);
    }
    __device__ __forceinline__ void norm2(float2 w) {
        df_fma(w.x, w.x, rh, rl);
        df_fma(w.y, w.y, rh, rl);
    }
    __device__ __forceinline__ double2 get() const {
        return make_double2((double)rh + (double)rl, (double)ih + (double)il);
    }
};

// Native arithmetic type of a vector element (float2 math for complex64 vectors).
__device__ __forceinline__ float2 to_vt(double2 v, const float2 *) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_vt(double2 v, const double2 *) { return v; }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return csub(a, b); }
template <class VT>
__device__ __forceinline__ VT vzero() {
    VT z;
    z.x = 0;
    z.y = 0;
    return z;
}

// ------------------------------------------------------------------ reduction stage 1

// Thread layout of the column kernels: CX lanes across columns (power of two <= 32),
// RY = 256 / CX rows in flight; block b of the grid owns rows [b*chunk, (b+1)*chunk).
struct RowSplit {
    int cx = 32, ry = 8, nrb = 1;
};

static RowSplit row_split(int64_t n, int64_t na, int num_sms) {
    RowSplit s;
    int cx = 1;
    while (cx < na && cx < 32) cx <<= 1;
    s.cx = cx;
    s.ry = 256 / cx;
    int64_t want = std::max<int64_t>(1, (n + 127) / 128);
    s.nrb = (int)std::min<int64_t>(want, (int64_t)2 * std::max(1, num_sms));
    return s;
}

constexpr int IG = 8;          // basis vectors per block in the projection kernels
constexpr int MAX_GROUP = 64;  // vectors per projection launch (partial buffer capacity)

enum { RED_CDOT = 0, RED_BILIN = 1, RED_NORM2 = 2 };

// partial[((i0+g)*na + c)*nrb + b] = sum over the block's rows of
//   RED_CDOT : conj(V_{i0+g}) w      RED_BILIN: V_{i0+g} w (no conjugation)
//   RED_NORM2: |w|^2 (nvec = 1, V unused)
// Grid: (row blocks, vector groups of IG, column chunks of cx).
template <class VT>
__global__ void __launch_bounds__(256) k_colpart(int64_t n, int64_t na, int nvec, int mode, const VT *__restrict__ V,
                                                 int64_t vstride, const VT *__restrict__ w, int cx, int ry, int nrb,
                                                 double2 *__restrict__ partial) {
    __shared__ double2 sm[IG][256];
    const int tx = threadIdx.x % cx, ty = threadIdx.x / cx;
    const int64_t chunk = (n + nrb - 1) / nrb;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    const int i0 = blockIdx.y * IG;
    const int ng = min(IG, nvec - i0);
    const int64_t c = (int64_t)blockIdx.z * cx + tx;
    Acc<VT> acc[IG];
#pragma unroll
    for (int g = 0; g < IG; ++g) acc[g].zero();
    if (c < na) {
        const VT *Vb = V + (int64_t)i0 * vstride;
        int64_t r = r0 + ty;
        for (; r + ry < r1; r += 2 * ry) {   // two rows per trip: more loads in flight
            const int64_t e0 = r * na + c, e1 = (r + ry) * na + c;
            const VT w0 = w[e0], w1 = w[e1];
            if (mode == RED_NORM2) {
                acc[0].norm2(w0);
                acc[0].norm2(w1);
            } else {
#pragma unroll
                for (int g = 0; g < IG; ++g) {
                    if (g < ng) {
                        const VT v0 = Vb[g * vstride + e0], v1 = Vb[g * vstride + e1];
                        if (mode == RED_CDOT) {
                            acc[g].cdot(v0, w0);
                            acc[g].cdot(v1, w1);
                        } else {
                            acc[g].bilin(v0, w0);
                            acc[g].bilin(v1, w1);
                        }
                    }
                }
            }
        }
        if (r < r1) {
            const int64_t e0 = r * na + c;
            const VT w0 = w[e0];
            if (mode == RED_NORM2) {
                acc[0].norm2(w0);
            } else {
#pragma unroll
                for (int g = 0; g < IG; ++g)
                    if (g < ng) {
                        const VT v0 = Vb[g * vstride + e0];
                        if (mode == RED_CDOT)
                            acc[g].cdot(v0, w0);
                        else
                            acc[g].bilin(v0, w0);
                    }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < IG; ++g) sm[g][threadIdx.x] = acc[g].get();
    __syncthreads();
    for (int st = ry >> 1; st > 0; st >>= 1) {
        if (ty < st)
            for (int g = 0; g < ng; ++g) sm[g][ty * cx + tx] = cadd(sm[g][ty * cx + tx], sm[g][(ty + st) * cx + tx]);
        __syncthreads();
    }
    if (ty == 0 && c < na)
        for (int g = 0; g < ng; ++g) partial[((int64_t)(i0 + g) * na + c) * nrb + blockIdx.x] = sm[g][tx];
}

static inline dim3 colpart_grid(int nrb, int nvec, int64_t na, int cx) {
    return dim3((unsigned)nrb, (unsigned)((nvec + IG - 1) / IG), (unsigned)((na + cx - 1) / cx));
}

// warp-level sum of the nrb partials of output o (block order fixed by the lane stride)
__device__ __forceinline__ double2 warp_sum_partials(const double2 *__restrict__ partial, int64_t o, int nrb,
                                                     int lane) {
    double2 s = czero();
    for (int b = lane; b < nrb; b += 32) s = cadd(s, partial[o * nrb + b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
    }
    return s;
}

// ------------------------------------------------------------------ GMRES device state

struct GmresDev {
    int m;
    int64_t na;      // active columns of the cycle
    double2 *H;      // [(m+1) * m][na]: H(i, j) of column c at (i * m + j) * na + c
    double *cs;      // [m][na]
    double2 *sn;     // [m][na]
    double2 *g;      // [m+1][na]
    double *target;  // [na] residual-estimate target of this cycle
    int *done;       // [na]
    int *jdone;      // [na] Arnoldi steps the column uses in this cycle
    int *iters;      // [na] Krylov iterations of the column in this cycle
};

// Givens QR update of column j of H for column c (complex rotations, real cosine).
__device__ void givens_step(const GmresDev &st, int64_t c, int j) {
    if (st.done[c]) return;
    const int m = st.m;
    const int64_t na = st.na;
    auto Hp = [&](int i, int jj) { return st.H + ((int64_t)i * m + jj) * na + c; };
    for (int i = 0; i < j; ++i) {
        const double cs = st.cs[(int64_t)i * na + c];
        const double2 sn = st.sn[(int64_t)i * na + c];
        const double2 a = *Hp(i, j), b = *Hp(i + 1, j);
        *Hp(i, j) = cadd(cscale(cs, a), cmul(sn, b));
        *Hp(i + 1, j) = csub(cscale(cs, b), cjmul(sn, a));
    }
    const double2 a = *Hp(j, j);
    const double hb = Hp(j + 1, j)->x;  // a norm: real, >= 0
    const double na_ = sqrt(cabs2(a));
    const double nu = sqrt(na_ * na_ + hb * hb);
    double cs;
    double2 sn, rdiag;
    if (nu == 0.0) {
        cs = 1.0;
        sn = czero();
        rdiag = a;
    } else if (na_ == 0.0) {
        cs = 0.0;
        sn = make_double2(1.0, 0.0);
        rdiag = make_double2(hb, 0.0);
    } else {
        const double2 ph = cscale(1.0 / na_, a);
        cs = na_ / nu;
        sn = cscale(hb / nu, ph);
        rdiag = cscale(nu, ph);
    }
    st.cs[(int64_t)j * na + c] = cs;
    st.sn[(int64_t)j * na + c] = sn;
    *Hp(j, j) = rdiag;
    *Hp(j + 1, j) = czero();
    const double2 gj = st.g[(int64_t)j * na + c];
    // g_{j+1} = -conj(sn) g_j,  g_j = cs g_j
    st.g[(int64_t)(j + 1) * na + c] = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
    st.g[(int64_t)j * na + c] = cscale(cs, gj);
    st.iters[c] += 1;
    const double res = sqrt(cabs2(st.g[(int64_t)(j + 1) * na + c]));
    if (res <= st.target[c] || hb == 0.0 || nu == 0.0) {
        st.done[c] = 1;
        st.jdone[c] = j + 1;
    }
}

enum { FIN_SET = 0, FIN_ADD = 1, FIN_NORM_GIVENS = 2, FIN_NORM = 3 };

// Stage 2 for GMRES: one warp per output (i, c), i < nvec.
//   FIN_SET        : out[i*ostride + c] = s
//   FIN_ADD        : out[i*ostride + c] += s; tmp[i*na + c] = s
//   FIN_NORM_GIVENS: tmp[c] = ||w||, H(j+1, j) = ||w||, Givens step of column j
//   FIN_NORM       : tmp[c] = (||v||, 0)
__global__ void __launch_bounds__(256) k_colfin(int64_t na, int nvec, int nrb, int mode,
                                                const double2 *__restrict__ partial, double2 *__restrict__ out,
                                                int64_t ostride, double2 *__restrict__ tmp, GmresDev st, int j) {
    const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (o >= (int64_t)nvec * na) return;
    const double2 s = warp_sum_partials(partial, o, nrb, lane);
    if (lane != 0) return;
    const int64_t i = o / na, c = o % na;
    if (mode == FIN_SET) {
        out[i * ostride + c] = s;
    } else if (mode == FIN_ADD) {
        out[i * ostride + c] = cadd(out[i * ostride + c], s);
        tmp[o] = s;
    } else if (mode == FIN_NORM_GIVENS) {
        const double2 hn = make_double2(sqrt(s.x), 0.0);
        tmp[c] = hn;
        st.H[((int64_t)(j + 1) * st.m + j) * na + c] = hn;
        givens_step(st, c, j);
    } else {
        tmp[c] = make_double2(sqrt(s.x), 0.0);
    }
}

// w -= sum_{i < nvec} coef[i*cstride + c] V_i   (one projection pass); one element per
// thread, eight independent partial sums so that eight basis loads are in flight.  The
// arithmetic is that of the vectors (FP32 for complex64 bases; the coefficients are the
// FP64 projections rounded to it).
template <class VT>
__global__ void __launch_bounds__(256) k_project(uint32_t total, uint32_t na, int nvec, const VT *__restrict__ V,
                                                 int64_t vstride, const double2 *__restrict__ coef, int64_t cstride,
                                                 VT *__restrict__ w) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t c = e % na;
    const VT *tag = nullptr;
    VT acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = vzero<VT>();
    int i = 0;
    for (; i + 8 <= nvec; i += 8) {
        VT v[8], h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            v[u] = V[(int64_t)(i + u) * vstride + e];
            h[u] = to_vt(coef[(int64_t)(i + u) * cstride + c], tag);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = vadd(acc[u], vmul(h[u], v[u]));
    }
    for (; i < nvec; ++i) acc[0] = vadd(acc[0], vmul(to_vt(coef[(int64_t)i * cstride + c], tag), V[(int64_t)i * vstride + e]));
    VT t = acc[0];
#pragma unroll
    for (int u = 1; u < 8; ++u) t = vadd(t, acc[u]);
    w[e] = vsub(w[e], t);
}

// ------------------------------------------------------------------ elementwise kernels
// (32-bit flat index e = r * na + c; callers guarantee n * na < 2^31)

// v <- v / h_c (zero for columns that are done: their later basis vectors are not used)
template <class VT>
__global__ void k_scale(uint32_t total, uint32_t na, VT *__restrict__ v, const double2 *__restrict__ h,
                        const int *__restrict__ done) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t c = e % na;
    const double hv = h[c].x;
    const double s = (done[c] || hv == 0.0) ? 0.0 : 1.0 / hv;
    VT x = v[e];
    x.x *= s;
    x.y *= s;
    v[e] = x;
}

// dst[r][k] = src[r][idx[k]]  (gather of active columns; src has ncol columns)
template <class TD, class TS>
__global__ void k_gather(uint32_t total, uint32_t na, int64_t ncol, const int *__restrict__ idx,
                         const TS *__restrict__ src, TD *__restrict__ dst) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t r = e / na, k = e % na;
    st2(dst + e, ld2(src + (int64_t)r * ncol + idx[k]));
}

// dst[r][idx[k]] += src[r][k]
__global__ void k_scatter_set(uint32_t total, uint32_t na, int64_t ncol, const int *__restrict__ idx,
                              const double2 *__restrict__ src, double2 *__restrict__ dst) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t r = e / na, k = e % na;
    dst[(int64_t)r * ncol + idx[k]] = src[e];
}

__global__ void k_scatter_add(uint32_t total, uint32_t na, int64_t ncol, const int *__restrict__ idx,
                              const double2 *__restrict__ src, double2 *__restrict__ dst) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t r = e / na, k = e % na;
    double2 *d = dst + (int64_t)r * ncol + idx[k];
    *d = cadd(*d, src[e]);
}

// r = B - Y (FP64)
__global__ void k_residual(uint32_t total, const double2 *__restrict__ B, const double2 *__restrict__ Y,
                           double2 *__restrict__ r) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < total) r[e] = csub(B[e], Y[e]);
}

// B[i][c] = R[i][col_dir[c]]
__global__ void k_make_b(uint32_t total, uint32_t cc, int ndir, const int *__restrict__ col_dir,
                         const double *__restrict__ R, double2 *__restrict__ B) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t i = e / cc, c = e % cc;
    B[e] = make_double2(R[(int64_t)i * ndir + col_dir[c]], 0.0);
}

// v0 = r / ||r|| (zero for columns marked done)
template <class VT>
__global__ void k_start_basis(uint32_t total, uint32_t na, const double2 *__restrict__ r,
                              const double2 *__restrict__ rnorm, const int *__restrict__ done, VT *__restrict__ v0) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t c = e % na;
    const double s = (done[c] || rnorm[c].x == 0.0) ? 0.0 : 1.0 / rnorm[c].x;
    st2(v0 + e, cscale(s, r[e]));
}

// d = sum_{l < jd_c} y_l V_l  (FP64)
template <class VT>
__global__ void k_combine(uint32_t total, uint32_t na, int jmax, const VT *__restrict__ V, int64_t vstride,
                          const double2 *__restrict__ y, const int *__restrict__ jdone, double2 *__restrict__ d) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t c = e % na;
    const int jd = min(jdone[c], jmax);
    const VT *tag = nullptr;
    VT s = vzero<VT>();
    for (int l = 0; l < jd; ++l) s = vadd(s, vmul(to_vt(y[(int64_t)l * na + c], tag), V[l * vstride + e]));
    d[e] = ld2(&s);
}

// per-column cycle set-up (done, targets, g0) from the residual norms of the active block
__global__ void k_cycle_cols(int64_t na, const double2 *__restrict__ rnorm, double inner_red,
                             const double *__restrict__ bnorm_a, double tol, GmresDev st) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= na) return;
    const double rn = rnorm[c].x;
    st.done[c] = (rn == 0.0) ? 1 : 0;
    st.jdone[c] = 0;
    st.iters[c] = 0;
    st.g[c] = make_double2(rn, 0.0);
    st.target[c] = fmax(0.5 * tol * bnorm_a[c], inner_red * rn);
}

// y = R^{-1} g on the first jd rows (R = rotated H); one thread per column
__global__ void k_backsolve(int64_t na, int jlast, GmresDev st, double2 *__restrict__ y) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= na) return;
    const int m = st.m;
    const int jd = st.done[c] ? st.jdone[c] : (jlast + 1);
    st.jdone[c] = jd;
    for (int l = jd - 1; l >= 0; --l) {
        double2 s = st.g[(int64_t)l * na + c];
        for (int k = l + 1; k < jd; ++k) s = csub(s, cmul(st.H[((int64_t)l * m + k) * na + c], y[(int64_t)k * na + c]));
        y[(int64_t)l * na + c] = cdiv(s, st.H[((int64_t)l * m + l) * na + c]);
    }
}

__global__ void k_set_z(int64_t cc, const double *__restrict__ col_omega, ShiftModel zm,
                        double2 *__restrict__ z) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cc) return;
    z[c] = z_eval(zm, col_omega[c]);
}

// ------------------------------------------------------------------ shared solver set-up

struct Common {
    wfq_geom *g = nullptr;
    cudaStream_t s = nullptr;
    int64_t n = 0, cc = 0;
    int num_sms = 1;
    DevBuf<double2> B, z, partial, bnorm, rnorm, tmp;
    DevBuf<double> R, dirs, omega;
    DevBuf<int> idx, coldir;
    // per-cycle compacted FP64 buffers (sized for all columns)
    DevBuf<double2> Ba, xa, ra, Ya, Ua, za;
    DevBuf<double> bnorm_a;
    std::vector<double> bn_h, res_h;   // ||B_c||, final relative residual per column
    bool residual_df = false;          // double-float D products in the true residual
    bool residual_exact = false;       // FP64 D products in the true residual (overrides residual_df)

    // A mixed solve on a geometry with no stored D takes its residuals from the double-float
    // product that regenerates D; where those hold a column's residual at a floor, the
    // residual can switch to D regenerated in FP64.
    bool can_tighten_residual() const {
        return residual_df && !residual_exact && !g->D64 && !g->Dfh && !g->Dsym && g->op == OP_WFQ;
    }

    int init(wfq_geom *geom, const SolveArgs &a, cudaStream_t stream) {
        g = geom;
        s = stream;
        n = g->n;
        cc = a.col_omega ? a.ncols : a.nfreq * a.ndir;
        std::vector<double> om_c(cc);
        std::vector<int> dir_c(cc);
        for (int64_t c = 0; c < cc; ++c) {
            om_c[c] = a.col_omega ? a.col_omega[c] : a.omega[c / a.ndir];
            dir_c[c] = a.col_dir ? a.col_dir[c] : (int)(c % a.ndir);
        }
        num_sms = g->ctx->num_sms;
        if ((double)n * (double)cc * 2.0 >= 2147483647.0)
            return fail(WFQ_EUNSUPPORTED, "n * columns too large for one block (>= 2^30)");
        wfq_ctx *ctx = g->ctx;
        const RowSplit rs = row_split(n, cc, num_sms);
        const size_t part = (size_t)rs.nrb * cc * MAX_GROUP;
        WFQ_TRY(B.alloc(ctx, n * cc, s));
        WFQ_TRY(z.alloc(ctx, cc, s));
        WFQ_TRY(partial.alloc(ctx, part, s));
        WFQ_TRY(bnorm.alloc(ctx, cc, s));
        WFQ_TRY(rnorm.alloc(ctx, cc, s));
        WFQ_TRY(tmp.alloc(ctx, (size_t)cc * MAX_GROUP, s));
        WFQ_TRY(R.alloc(ctx, n * a.ndir, s));
        WFQ_TRY(dirs.alloc(ctx, 3 * a.ndir, s));
        WFQ_TRY(omega.alloc(ctx, cc, s));
        WFQ_TRY(idx.alloc(ctx, cc, s));
        WFQ_TRY(coldir.alloc(ctx, cc, s));
        WFQ_TRY(Ba.alloc(ctx, n * cc, s));
        WFQ_TRY(xa.alloc(ctx, n * cc, s));
        WFQ_TRY(ra.alloc(ctx, n * cc, s));
        WFQ_TRY(Ya.alloc(ctx, n * cc, s));
        WFQ_TRY(Ua.alloc(ctx, n * cc, s));
        WFQ_TRY(za.alloc(ctx, cc, s));
        WFQ_TRY(bnorm_a.alloc(ctx, cc, s));
        WFQ_CUDA(cudaMemcpyAsync(dirs.ptr, a.dirs, sizeof(double) * 3 * a.ndir, cudaMemcpyHostToDevice, s));
        WFQ_CUDA(cudaMemcpyAsync(omega.ptr, om_c.data(), sizeof(double) * cc, cudaMemcpyHostToDevice, s));
        WFQ_CUDA(cudaMemcpyAsync(coldir.ptr, dir_c.data(), sizeof(int) * cc, cudaMemcpyHostToDevice, s));
        k_set_z<<<nblocks(cc), 256, 0, s>>>(cc, omega.ptr, shift_model(g), z.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        WFQ_TRY(launch_rhs(g, a.ndir, dirs.ptr, a.E0, R.ptr, s));
        k_make_b<<<nblocks(n * cc), 256, 0, s>>>((uint32_t)(n * cc), (uint32_t)cc, a.ndir, coldir.ptr, R.ptr, B.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        WFQ_TRY(colnorm(B.ptr, cc, bnorm.ptr));
        bn_h.assign(cc, 0.0);
        res_h.assign(cc, 0.0);
        std::vector<double2> t(cc);
        WFQ_CUDA(cudaMemcpyAsync(t.data(), bnorm.ptr, sizeof(double2) * cc, cudaMemcpyDeviceToHost, s));
        WFQ_CUDA(cudaStreamSynchronize(s));
        for (int64_t c = 0; c < cc; ++c) bn_h[c] = t[c].x;
        return WFQ_OK;
    }

    // out[c].x = ||v_c|| for a block of na columns (FP64 vectors)
    int colnorm(const double2 *v, int64_t na, double2 *out) {
        const RowSplit rs = row_split(n, na, num_sms);
        k_colpart<double2><<<colpart_grid(rs.nrb, 1, na, rs.cx), 256, 0, s>>>(n, na, 1, RED_NORM2, nullptr, 0, v, rs.cx,
                                                                              rs.ry, rs.nrb, partial.ptr); note_launch();
        GmresDev dummy{};
        k_colfin<<<nblocks(na * 32), 256, 0, s>>>(na, 1, rs.nrb, FIN_NORM, partial.ptr, nullptr, 0, out, dummy, 0); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }

    // Upload the active column list and gather B, z, ||B|| for it.
    int select(const std::vector<int> &act) {
        const int64_t na = (int64_t)act.size();
        WFQ_CUDA(cudaMemcpyAsync(idx.ptr, act.data(), sizeof(int) * na, cudaMemcpyHostToDevice, s));
        const uint32_t tot = (uint32_t)(n * na);
        k_gather<double2, double2><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, cc, idx.ptr, B.ptr, Ba.ptr); note_launch();
        k_gather<double2, double2><<<nblocks(na), 256, 0, s>>>((uint32_t)na, (uint32_t)na, cc, idx.ptr, z.ptr, za.ptr); note_launch();
        std::vector<double> bn(na);
        for (int64_t k = 0; k < na; ++k) bn[k] = bn_h[act[k]];
        WFQ_CUDA(cudaMemcpyAsync(bnorm_a.ptr, bn.data(), sizeof(double) * na, cudaMemcpyHostToDevice, s));
        WFQ_CUDA(cudaStreamSynchronize(s));   // bn lives on this stack frame
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }

    // ra = Ba - (A - z I) xa in FP64 over the na active columns (xa gathered from x);
    // rnorm[k] = ||ra_k||.
    int true_residual(const double2 *x, int64_t na) {
        KScope ks(g->ctx, WFQ_KT_RESIDUAL, s);
        const uint32_t tot = (uint32_t)(n * na);
        k_gather<double2, double2><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, cc, idx.ptr, x, xa.ptr); note_launch();
        if (residual_df && !residual_exact)
            WFQ_TRY(d_apply_df(g, na, xa.ptr, Ua.ptr, s));
        else
            WFQ_TRY(d_apply_fp64(g, na, xa.ptr, Ua.ptr, s));
        WFQ_TRY(sparse_shift_fp64(g, na, Ua.ptr, xa.ptr, za.ptr, Ya.ptr, s));
        k_residual<<<nblocks(tot), 256, 0, s>>>(tot, Ba.ptr, Ya.ptr, ra.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return colnorm(ra.ptr, na, rnorm.ptr);
    }

    // As true_residual for all cc columns in order (after select of 0..cc-1), with the
    // product D x supplied (dx, n x cc) instead of computed here.
    int residual_given_dx(const double2 *x, const double2 *dx) {
        KScope ks(g->ctx, WFQ_KT_RESIDUAL, s);
        const uint32_t tot = (uint32_t)(n * cc);
        WFQ_TRY(sparse_shift_fp64(g, cc, dx, x, za.ptr, Ya.ptr, s));
        k_residual<<<nblocks(tot), 256, 0, s>>>(tot, Ba.ptr, Ya.ptr, ra.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return colnorm(ra.ptr, cc, rnorm.ptr);
    }

    // Narrow the active set from `act` to `keep` (a subset, same order): the residual
    // block ra and its norms are gathered from the wider block (no new FP64 product),
    // then B, z and ||B|| are re-gathered for the new list.
    int narrow(std::vector<int> &act, const std::vector<int> &keep) {
        const int64_t na_old = (int64_t)act.size(), na = (int64_t)keep.size();
        std::vector<int> sub;
        sub.reserve(na);
        for (int64_t k = 0, q = 0; k < na_old && q < na; ++k)
            if (act[k] == keep[q]) {
                sub.push_back((int)k);
                ++q;
            }
        WFQ_CUDA(cudaMemcpyAsync(idx.ptr, sub.data(), sizeof(int) * na, cudaMemcpyHostToDevice, s));
        const uint32_t tot = (uint32_t)(n * na);
        k_gather<double2, double2><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, na_old, idx.ptr, ra.ptr, Ya.ptr); note_launch();
        k_gather<double2, double2><<<nblocks(na), 256, 0, s>>>((uint32_t)na, (uint32_t)na, na_old, idx.ptr, rnorm.ptr, tmp.ptr); note_launch();
        WFQ_CUDA(cudaMemcpyAsync(ra.ptr, Ya.ptr, sizeof(double2) * tot, cudaMemcpyDeviceToDevice, s));
        WFQ_CUDA(cudaMemcpyAsync(rnorm.ptr, tmp.ptr, sizeof(double2) * na, cudaMemcpyDeviceToDevice, s));
        WFQ_CUDA(cudaStreamSynchronize(s));   // sub lives on this stack frame
        act = keep;
        return select(act);
    }

    // ra = Ba - (A - z I) xa with the mixed operator (xa rounded to complex64): the restart
    // residual of a cycle whose columns are all still far from the tolerance, where its
    // ~1e-6 relative error is irrelevant.  Never used to declare convergence.
    int mixed_residual(const double2 *x, int64_t na, float2 *xs, float2 *u32, float2 *y32, void *scratch) {
        KScope ks(g->ctx, WFQ_KT_RESIDUAL, s);
        const uint32_t tot = (uint32_t)(n * na);
        k_gather<float2, double2><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, cc, idx.ptr, x, xs); note_launch();
        WFQ_TRY(d_apply_mixed(g, na, xs, u32, scratch, s));
        WFQ_TRY(sparse_shift_fp32(g, na, u32, xs, za.ptr, y32, s));
        k_gather<double2, float2><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, na, idx_identity(na), y32, Ya.ptr); note_launch();
        k_residual<<<nblocks(tot), 256, 0, s>>>(tot, Ba.ptr, Ya.ptr, ra.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return colnorm(ra.ptr, na, rnorm.ptr);
    }

    // identity column map 0..na-1 (for widening a complex64 block to FP64)
    DevBuf<int> ident;
    int64_t ident_n = 0;
    const int *idx_identity(int64_t na) {
        if (ident_n < na) {
            std::vector<int> h(cc);
            for (int64_t k = 0; k < cc; ++k) h[k] = (int)k;
            if (!ident.ptr) ident.alloc(g->ctx, cc, s);
            cudaMemcpyAsync(ident.ptr, h.data(), sizeof(int) * cc, cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);
            ident_n = cc;
        }
        return ident.ptr;
    }

    // Host copy of rnorm for the na active columns; records each column's relative
    // residual and returns the columns that have not reached tol.
    int classify(const std::vector<int> &act, double tol, std::vector<int> &still) {
        const int64_t na = (int64_t)act.size();
        std::vector<double2> rn(na);
        WFQ_CUDA(cudaMemcpyAsync(rn.data(), rnorm.ptr, sizeof(double2) * na, cudaMemcpyDeviceToHost, s));
        WFQ_TRY(check_device_error(g->ctx, s));
        still.clear();
        for (int64_t k = 0; k < na; ++k) {
            const int c = act[k];
            const double rel = bn_h[c] > 0.0 ? rn[k].x / bn_h[c] : 0.0;
            res_h[c] = rel;
            if (!(rel <= tol)) still.push_back(c);
        }
        return WFQ_OK;
    }
};

static int finish_stats(const SolveArgs &a, const Common &cm, const std::vector<int> &iters, int cycles,
                        const std::vector<int> &breakdown) {
    bool all = true, brk_any = false;
    for (int64_t c = 0; c < cm.cc; ++c) {
        const bool ok = cm.res_h[c] <= a.rel_tol;
        const bool brk = !breakdown.empty() && breakdown[c];
        all = all && ok;
        brk_any = brk_any || (brk && !ok);
        if (a.stats) {
            wfq_stats &st = a.stats[c];
            st.iters = iters[c];
            st.restarts = std::max(0, cycles - 1);
            st.refinements = (a.prec == WFQ_PREC_MIXED) ? std::max(0, cycles - 1) : 0;
            st.rel_residual = cm.res_h[c];
            st.rmse = cm.res_h[c] * cm.bn_h[c] / std::sqrt((double)cm.n);
            st.status = ok ? WFQ_OK : (brk ? WFQ_EBREAKDOWN : WFQ_ENOCONV);
        }
    }
    if (all) return WFQ_OK;
    if (brk_any) return fail(WFQ_EBREAKDOWN, "QMR breakdown (rho or sigma = 0) without convergence");
    return fail(WFQ_ENOCONV, "iteration limit reached before rel_tol in some column");
}

// ------------------------------------------------------------------ GMRES

// Per-column outcome of one GMRES run, for the caller that continues it.
struct GmresOut {
    std::vector<int> escalate;   // mixed solve: columns whose refinement stagnated
    std::vector<double> res;     // final relative residual (FP64 true residual)
    std::vector<int> iters;      // Krylov iterations
    int cycles = 0;
};

// A column of the mixed solve leaves it, to be finished in plain FP64, when its FP64 true
// residual shrank by less than STAGNATION_RATIO in each of STAGNATION_CYCLES consecutive
// refinement cycles while the inner solve had reached its own target (GMRES: the mixed
// operator's residual estimate below FLOOR_GAP times the true residual; QMR: the column
// converged in the inner run): the operator error times the conditioning of A - zI is not
// small, or the residual sits at the rounding floor of the double-float residual.  A cycle
// that ended with the inner solve short of its target shows slow Krylov convergence, which
// FP64 iterations would repeat at many times the cost: such a column escalates only after
// SLOW_CYCLES consecutive slow cycles.
constexpr double STAGNATION_RATIO = 0.5;
constexpr int STAGNATION_CYCLES = 2;
constexpr double FLOOR_GAP = 0.25;
constexpr int SLOW_CYCLES = 20;
constexpr int FLOOR_CYCLES = 5;

template <class VT>
static int gmres_impl(wfq_geom *g, const SolveArgs &a, cudaStream_t s, GmresOut *out) {
    Common cm;
    WFQ_TRY(cm.init(g, a, s));
    const int64_t n = cm.n, cc = cm.cc;
    const bool mixed = (a.prec == WFQ_PREC_MIXED);
    cm.residual_df = mixed;
    int m = a.m > 0 ? std::min(a.m, a.max_iter) : a.max_iter;
    m = std::max(1, m);
    wfq_ctx *ctx = g->ctx;

    DevBuf<VT> V;
    DevBuf<double2> H, sn, gv, y, hn;
    DevBuf<double> cs, target;
    DevBuf<int> done, jdone, iters;
    DevBuf<float2> U32;
    DevBuf<unsigned char> scratch;
    WFQ_TRY(V.alloc(ctx, (size_t)(m + 1) * n * cc, s));
    WFQ_TRY(H.alloc(ctx, (size_t)(m + 1) * m * cc, s));
    WFQ_TRY(sn.alloc(ctx, (size_t)m * cc, s));
    WFQ_TRY(gv.alloc(ctx, (size_t)(m + 1) * cc, s));
    WFQ_TRY(y.alloc(ctx, (size_t)m * cc, s));
    WFQ_TRY(hn.alloc(ctx, (size_t)cc, s));
    WFQ_TRY(cs.alloc(ctx, (size_t)m * cc, s));
    WFQ_TRY(target.alloc(ctx, cc, s));
    WFQ_TRY(done.alloc(ctx, cc, s));
    WFQ_TRY(jdone.alloc(ctx, cc, s));
    WFQ_TRY(iters.alloc(ctx, cc, s));
    if (mixed) {
        WFQ_TRY(U32.alloc(ctx, n * cc, s));
        WFQ_TRY(scratch.alloc(ctx, mixed_scratch_bytes(g, cc), s));
    }
    if (!a.warm) WFQ_CUDA(cudaMemsetAsync(a.q, 0, sizeof(double2) * n * cc, s));
    const double inner_red = mixed ? 1e-6 : 0.0;
    std::vector<int> act(cc), still;
    for (int64_t c = 0; c < cc; ++c) act[c] = (int)c;
    std::vector<int> iters_h(cc, 0), it_a, done_h;
    DevBuf<float2> xs32, y32;
    if (mixed) {
        WFQ_TRY(xs32.alloc(ctx, n * cc, s));
        WFQ_TRY(y32.alloc(ctx, n * cc, s));
    }
    int total = 0, cycles = 0;
    WFQ_TRY(cm.select(act));
    if (a.warm) {
        WFQ_TRY(cm.true_residual(a.q, cc));
    } else {   // x0 = 0: the first residual is R itself
        WFQ_CUDA(cudaMemcpyAsync(cm.ra.ptr, cm.Ba.ptr, sizeof(double2) * n * cc, cudaMemcpyDeviceToDevice, s));
        WFQ_TRY(cm.colnorm(cm.ra.ptr, cc, cm.rnorm.ptr));
    }
    bool exact = true;   // the current residual block was computed to FP64 accuracy
    std::vector<double2> g_h;
    std::vector<int> jd_h;
    std::vector<double> prev_exact(cc, -1.0);   // last FP64 relative residual per column
    std::vector<int> esc, flat_cycles(cc, 0), slow_cycles(cc, 0);
    std::vector<double> inner_est(cc, -1.0);   // mixed: last cycle's inner residual estimate (absolute)

    for (;;) {
        if (exact) {
            WFQ_TRY(cm.classify(act, a.rel_tol, still));
            if (mixed && out) {
                std::vector<int> keep;
                keep.reserve(still.size());
                bool tighten = false;
                for (int c : still) {
                    const bool slow = prev_exact[c] >= 0.0 && cm.res_h[c] > STAGNATION_RATIO * prev_exact[c];
                    const bool floor = inner_est[c] >= 0.0 && inner_est[c] < FLOOR_GAP * cm.res_h[c] * cm.bn_h[c];
                    flat_cycles[c] = slow && floor ? flat_cycles[c] + 1 : 0;
                    slow_cycles[c] = slow ? slow_cycles[c] + 1 : 0;
                    prev_exact[c] = cm.res_h[c];
                    if (flat_cycles[c] >= STAGNATION_CYCLES && cm.can_tighten_residual()) tighten = true;
                    if (flat_cycles[c] >= STAGNATION_CYCLES || slow_cycles[c] >= SLOW_CYCLES)
                        esc.push_back(c);
                    else
                        keep.push_back(c);
                }
                if (tighten) {
                    // the floor is the residual's: recompute it with D in FP64 and carry on
                    // in mixed precision with every column of this cycle
                    esc.resize(esc.size() - (still.size() - keep.size()));
                    cm.residual_exact = true;
                    std::fill(flat_cycles.begin(), flat_cycles.end(), 0);
                    std::fill(slow_cycles.begin(), slow_cycles.end(), 0);
                    std::fill(prev_exact.begin(), prev_exact.end(), -1.0);
                    trace("gmres(%d) mixed cycle %d: residual floor of the regenerated double-float D; residuals "
                          "from D in FP64 from here", m, cycles);
                    WFQ_TRY(cm.true_residual(a.q, (int64_t)act.size()));
                    continue;
                }
                still.swap(keep);
            } else if (!mixed) {
                // FP64: a column within 100 x tol whose true residual fell by less than 10% in
                // each of FLOOR_CYCLES consecutive cycles sits at the rounding floor of its
                // residual; it stops (not converged) instead of cycling to max_iter.
                std::vector<int> keep;
                keep.reserve(still.size());
                for (int c : still) {
                    const bool flat = prev_exact[c] >= 0.0 && cm.res_h[c] > 0.9 * prev_exact[c] &&
                                      cm.res_h[c] < 100.0 * a.rel_tol;
                    flat_cycles[c] = flat ? flat_cycles[c] + 1 : 0;
                    prev_exact[c] = cm.res_h[c];
                    if (flat_cycles[c] < FLOOR_CYCLES) keep.push_back(c);
                }
                still.swap(keep);
            }
            if (trace_on()) {
                double worst = 0.0;
                for (int c : act) worst = std::max(worst, cm.res_h[c]);
                trace("gmres(%d) %s cycle %d: %zu of %zu columns active, %zu escalated, %d steps, max true "
                      "rel. residual %.3e", m, mixed ? "mixed" : "fp64", cycles, still.size(), act.size(), esc.size(),
                      total, worst);
            }
            if (still.empty() || total >= a.max_iter) break;
            if (still.size() != act.size()) WFQ_TRY(cm.narrow(act, still));
        } else if (total >= a.max_iter) {
            WFQ_TRY(cm.true_residual(a.q, (int64_t)act.size()));   // final statistics are exact
            WFQ_TRY(cm.classify(act, a.rel_tol, still));
            break;
        }
        const int64_t na = (int64_t)act.size();
        // ---- one restart cycle on the na active columns
        const uint32_t tot = (uint32_t)(n * na);
        const int64_t vstride = n * na;
        GmresDev st{m, na, H.ptr, cs.ptr, sn.ptr, gv.ptr, target.ptr, done.ptr, jdone.ptr, iters.ptr};
        WFQ_CUDA(cudaMemsetAsync(H.ptr, 0, sizeof(double2) * (m + 1) * m * na, s));
        k_cycle_cols<<<nblocks(na), 256, 0, s>>>(na, cm.rnorm.ptr, inner_red, cm.bnorm_a.ptr, a.rel_tol, st); note_launch();
        k_start_basis<VT><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, cm.ra.ptr, cm.rnorm.ptr, done.ptr, V.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        const RowSplit rs = row_split(n, na, cm.num_sms);
        int jlast = -1;
        done_h.assign(na, 0);
        for (int j = 0; j < m && total < a.max_iter; ++j) {
            VT *vj = V.ptr + (int64_t)j * vstride;
            VT *w = V.ptr + (int64_t)(j + 1) * vstride;
            if (mixed) {
                WFQ_TRY(d_apply_mixed(g, na, reinterpret_cast<const float2 *>(vj), U32.ptr, scratch.ptr, s));
                WFQ_TRY(sparse_shift_fp32(g, na, U32.ptr, reinterpret_cast<const float2 *>(vj), cm.za.ptr,
                                          reinterpret_cast<float2 *>(w), s));
            } else {
                WFQ_TRY(solver_fp64_product(g, na, reinterpret_cast<const double2 *>(vj), cm.Ua.ptr, s));
                WFQ_TRY(sparse_shift_fp64(g, na, cm.Ua.ptr, reinterpret_cast<const double2 *>(vj), cm.za.ptr,
                                          reinterpret_cast<double2 *>(w), s));
            }
            KScope ko(g->ctx, WFQ_KT_ORTHO, s);
            // two classical Gram-Schmidt passes against V_0..V_j (groups of <= 64 vectors)
            for (int pass = 0; pass < 2; ++pass) {
                for (int i0 = 0; i0 <= j; i0 += MAX_GROUP) {
                    const int nv = std::min(MAX_GROUP, j + 1 - i0);
                    k_colpart<VT><<<colpart_grid(rs.nrb, nv, na, rs.cx), 256, 0, s>>>(
                        n, na, nv, RED_CDOT, V.ptr + (int64_t)i0 * vstride, vstride, w, rs.cx, rs.ry, rs.nrb,
                        cm.partial.ptr); note_launch();
                    double2 *hcol = H.ptr + ((int64_t)i0 * m + j) * na;
                    k_colfin<<<nblocks((int64_t)nv * na * 32), 256, 0, s>>>(na, nv, rs.nrb, pass == 0 ? FIN_SET : FIN_ADD,
                                                                           cm.partial.ptr, hcol, (int64_t)m * na,
                                                                           cm.tmp.ptr, st, j); note_launch();
                    const double2 *coef = pass == 0 ? hcol : cm.tmp.ptr;
                    const int64_t cstride = pass == 0 ? (int64_t)m * na : na;
                    k_project<VT><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, nv, V.ptr + (int64_t)i0 * vstride,
                                                               vstride, coef, cstride, w); note_launch();
                }
            }
            k_colpart<VT><<<colpart_grid(rs.nrb, 1, na, rs.cx), 256, 0, s>>>(n, na, 1, RED_NORM2, nullptr, 0, w, rs.cx,
                                                                             rs.ry, rs.nrb, cm.partial.ptr); note_launch();
            k_colfin<<<nblocks(na * 32), 256, 0, s>>>(na, 1, rs.nrb, FIN_NORM_GIVENS, cm.partial.ptr, nullptr, 0,
                                                      hn.ptr, st, j); note_launch();
            k_scale<VT><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, w, hn.ptr, done.ptr); note_launch();
            WFQ_CUDA(cudaGetLastError());
            ++total;
            jlast = j;
            WFQ_CUDA(cudaMemcpyAsync(done_h.data(), done.ptr, sizeof(int) * na, cudaMemcpyDeviceToHost, s));
            WFQ_CUDA(cudaStreamSynchronize(s));
            if (std::all_of(done_h.begin(), done_h.end(), [](int v) { return v != 0; })) break;
        }
        if (jlast >= 0) {
            // one thread per column, a serial FP64 chain each: spread over many SMs (few FP64
            // units per SM on GB300)
            k_backsolve<<<nblocks(na, 4), 4, 0, s>>>(na, jlast, st, y.ptr); note_launch();
            k_combine<VT><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, jlast + 1, V.ptr, vstride, y.ptr, jdone.ptr,
                                                       cm.Ya.ptr); note_launch();
            k_scatter_add<<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, cc, cm.idx.ptr, cm.Ya.ptr, a.q); note_launch();
            WFQ_CUDA(cudaGetLastError());
        }
        it_a.assign(na, 0);
        WFQ_CUDA(cudaMemcpyAsync(it_a.data(), iters.ptr, sizeof(int) * na, cudaMemcpyDeviceToHost, s));
        WFQ_CUDA(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < na; ++k) iters_h[act[k]] += it_a[k];
        ++cycles;
        // Next residual.  Mixed solves whose columns all ended this cycle with a residual
        // estimate above 1e-3 ||R|| restart from the mixed-operator residual; otherwise (and
        // always for FP64 solves) from the FP64-accurate true residual, which alone decides
        // convergence.
        bool far = false;
        if (mixed && jlast >= 0) {
            g_h.resize((size_t)(m + 1) * na);
            jd_h.resize(na);
            WFQ_CUDA(cudaMemcpyAsync(g_h.data(), gv.ptr, sizeof(double2) * (m + 1) * na, cudaMemcpyDeviceToHost, s));
            WFQ_CUDA(cudaMemcpyAsync(jd_h.data(), jdone.ptr, sizeof(int) * na, cudaMemcpyDeviceToHost, s));
            WFQ_CUDA(cudaStreamSynchronize(s));
            far = true;
            for (int64_t k = 0; k < na; ++k) {
                const double2 gk = g_h[(size_t)jd_h[k] * na + k];
                const double est = std::sqrt(gk.x * gk.x + gk.y * gk.y);
                inner_est[act[k]] = est;
                if (!(est > 1e-3 * cm.bn_h[act[k]])) far = false;
            }
        }
        if (far) {
            WFQ_TRY(cm.mixed_residual(a.q, na, xs32.ptr, U32.ptr, y32.ptr, scratch.ptr));
            exact = false;
            trace("gmres(%d) mixed cycle %d: all %lld columns above 1e-3 |R|, mixed-operator residual", m, cycles,
                  (long long)na);
        } else {
            WFQ_TRY(cm.true_residual(a.q, na));
            exact = true;
        }
    }
    if (out) {
        std::sort(esc.begin(), esc.end());
        out->escalate = esc;
        out->res = cm.res_h;
        out->iters = iters_h;
        out->cycles = cycles;
    }
    return finish_stats(a, cm, iters_h, cycles, {});
}

size_t solve_footprint(const wfq_geom *g, int64_t cc, int m, int prec) {
    const size_t n = (size_t)g->n, nc = n * (size_t)cc;
    const bool mixed = (prec == WFQ_PREC_MIXED);
    const size_t vt = mixed ? sizeof(float2) : sizeof(double2);
    size_t b = (size_t)(m + 1) * nc * vt;                       // Krylov basis
    b += 8 * nc * sizeof(double2);                              // B, FP64 active blocks, output
    b += (size_t)(m + 2) * (size_t)(m + 1) * cc * 48;           // Hessenberg, rotations
    b += (size_t)std::min<int64_t>((int64_t)(n + 127) / 128, 304) * cc * 64 * sizeof(double2);  // partials
    if (mixed) b += 3 * nc * sizeof(float2) + (size_t)round_up(2 * cc, 32) * (size_t)g->npad * 4;
    return b;
}

// Continue the columns `cols` of a solve from their iterate in a.q: block GMRES(m) at
// precision `prec` (mixed continuations that stall finish in FP64), warm-started; their q
// columns and statistics are replaced.  `res` / `iters`: relative residual and Krylov
// steps so far of every column (the others keep their state).
static int continue_columns(wfq_geom *g, const SolveArgs &a, const std::vector<int> &cols,
                            const std::vector<double> &res, const std::vector<int> &iters, int prec, int m,
                            cudaStream_t s) {
    const int64_t ne = (int64_t)cols.size(), n = g->n, cc = (int64_t)res.size();
    trace("continuing %lld of %lld columns by GMRES(%d) at %s", (long long)ne, (long long)cc, m,
          prec == WFQ_PREC_MIXED ? "mixed precision" : "FP64");
    int used = 0;
    for (int c : cols) used = std::max(used, iters[c]);
    if (a.max_iter - used < 1) return fail(WFQ_ENOCONV, "iteration limit reached before rel_tol in some column");
    std::vector<double> om(ne);
    std::vector<int> dir(ne);
    for (int64_t k = 0; k < ne; ++k) {
        const int c = cols[k];
        om[k] = a.col_omega ? a.col_omega[c] : a.omega[c / a.ndir];
        dir[k] = a.col_dir ? a.col_dir[c] : c % a.ndir;
    }
    DevBuf<double2> q2;
    DevBuf<int> idx;
    WFQ_TRY(q2.alloc(g->ctx, n * ne, s));
    WFQ_TRY(idx.alloc(g->ctx, ne, s));
    WFQ_CUDA(cudaMemcpyAsync(idx.ptr, cols.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, s));
    const uint32_t tot = (uint32_t)(n * ne);
    k_gather<double2, double2><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)ne, cc, idx.ptr, a.q, q2.ptr); note_launch();
    WFQ_CUDA(cudaGetLastError());
    std::vector<wfq_stats> st2(ne);
    SolveArgs b = a;
    b.col_omega = om.data();
    b.col_dir = dir.data();
    b.ncols = ne;
    b.q = q2.ptr;
    b.stats = st2.data();
    b.prec = prec;
    b.m = m;
    b.warm = true;
    b.max_iter = a.max_iter - used;
    const int rc2 = solve_gmres(g, b, s);
    if (rc2 != WFQ_OK && rc2 != WFQ_ENOCONV) return rc2;
    k_scatter_set<<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)ne, cc, idx.ptr, q2.ptr, a.q); note_launch();
    WFQ_CUDA(cudaGetLastError());
    WFQ_CUDA(cudaStreamSynchronize(s));   // idx, q2 and om/dir are released on return
    std::vector<char> cont(cc, 0);
    for (int c : cols) cont[c] = 1;
    bool all = true;
    for (int64_t c = 0; c < cc; ++c) all = all && (cont[c] || res[c] <= a.rel_tol);
    for (int64_t k = 0; k < ne; ++k) {
        all = all && st2[k].status == WFQ_OK;
        if (a.stats) {
            wfq_stats &st = a.stats[cols[k]];
            st.iters = iters[cols[k]] + st2[k].iters;
            st.restarts += st2[k].restarts + 1;
            st.refinements += st2[k].refinements;
            st.rel_residual = st2[k].rel_residual;
            st.rmse = st2[k].rmse;
            st.status = st2[k].status;
        }
    }
    if (all) {
        set_error("");   // an earlier stage's non-convergence message no longer applies
        return WFQ_OK;
    }
    return fail(WFQ_ENOCONV, "iteration limit reached before rel_tol in some column");
}

int finish_columns(wfq_geom *g, const SolveArgs &a, const std::vector<int> &iters, int m, const double2 *dq,
                   cudaStream_t s) {
    Common cm;
    WFQ_TRY(cm.init(g, a, s));
    cm.residual_df = true;
    std::vector<int> act(cm.cc), still;
    for (int64_t c = 0; c < cm.cc; ++c) act[c] = (int)c;
    WFQ_TRY(cm.select(act));
    if (dq)
        WFQ_TRY(cm.residual_given_dx(a.q, dq));
    else
        WFQ_TRY(cm.true_residual(a.q, cm.cc));
    WFQ_TRY(cm.classify(act, a.rel_tol, still));
    if (a.stats)
        for (int64_t c = 0; c < cm.cc; ++c) {
            wfq_stats &st = a.stats[c];
            st.iters = iters[c];
            st.restarts = 0;
            st.refinements = 0;
            st.rel_residual = cm.res_h[c];
            st.rmse = cm.res_h[c] * cm.bn_h[c] / std::sqrt((double)cm.n);
            st.status = cm.res_h[c] <= a.rel_tol ? WFQ_OK : WFQ_ENOCONV;
        }
    if (still.empty()) return WFQ_OK;
    return continue_columns(g, a, still, cm.res_h, iters, a.prec, m, s);
}

int solve_gmres(wfq_geom *g, const SolveArgs &a, cudaStream_t s) {
    if (a.prec != WFQ_PREC_MIXED) return gmres_impl<double2>(g, a, s, nullptr);
    GmresOut o1;
    const int rc = gmres_impl<float2>(g, a, s, &o1);
    if (o1.escalate.empty() || (rc != WFQ_OK && rc != WFQ_ENOCONV)) return rc;
    // the columns whose mixed refinement stalled finish in plain FP64 from the mixed
    // iterate: where ||A|| ||x|| / ||R|| is large (low frequencies on large flakes) the
    // double-float residual's ~1e-14 relative error already sits near the 1e-8 bar
    return continue_columns(g, a, o1.escalate, o1.res, o1.iters, WFQ_PREC_FP64, a.m, s);
}

// ------------------------------------------------------------------ QMR

struct QmrDev {
    int64_t na;
    double2 *rho, *sigma, *alpha, *beta;
    double *tau, *theta_old, *c2;   // c2: c^2 of the current step
    double2 *cd, *ca;               // d <- cd d + ca p
    double *target;
    int *done, *iters, *breakdown;
};

enum { QF_SIGMA = 0, QF_RNORM = 1, QF_SNORM = 2, QF_RHO = 3, QF_START = 4 };

// Stage 2 for QMR: one warp per active column, then the per-column scalar update.
__global__ void __launch_bounds__(256) k_qmr_fin(int64_t na, int nrb, int kind, const double2 *__restrict__ partial,
                                                 QmrDev q) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= na) return;
    const double2 s = warp_sum_partials(partial, c, nrb, lane);
    if (lane != 0) return;
    const bool dn = q.done[c] != 0;
    if (kind == QF_SIGMA) {
        q.sigma[c] = s;
        if (dn) {
            q.alpha[c] = czero();
        } else if (s.x == 0.0 && s.y == 0.0) {
            q.breakdown[c] = 1;
            q.done[c] = 1;
            q.alpha[c] = czero();
        } else {
            q.alpha[c] = cdiv(q.rho[c], s);
        }
    } else if (kind == QF_RNORM) {
        // smoothing weights from the BCG residual norm: theta = ||r||/tau, c^2 = 1/(1+theta^2)
        const double rn = sqrt(s.x);
        if (dn) {
            q.cd[c] = czero();
            q.ca[c] = czero();
            q.c2[c] = 0.0;
        } else {
            const double th = rn / q.tau[c];
            const double c2 = 1.0 / (1.0 + th * th);
            q.cd[c] = make_double2(c2 * q.theta_old[c] * q.theta_old[c], 0.0);
            q.ca[c] = cscale(c2, q.alpha[c]);
            q.c2[c] = c2;
            q.tau[c] = q.tau[c] * th * sqrt(c2);
            q.theta_old[c] = th;
        }
    } else if (kind == QF_SNORM) {
        if (!dn) {
            q.iters[c] += 1;
            if (sqrt(s.x) <= q.target[c]) q.done[c] = 1;
        }
    } else if (kind == QF_RHO) {
        if (dn) {
            q.beta[c] = czero();
        } else if (s.x == 0.0 && s.y == 0.0) {
            q.breakdown[c] = 1;
            q.done[c] = 1;
            q.beta[c] = czero();
        } else {
            q.beta[c] = cdiv(s, q.rho[c]);
            q.rho[c] = s;
        }
    } else {  // QF_START: rho = r^T D r of the restart residual
        q.rho[c] = s;
        if (!dn && s.x == 0.0 && s.y == 0.0) {
            q.breakdown[c] = 1;
            q.done[c] = 1;
        }
    }
}

template <class VT>
__global__ void k_qmr_r(uint32_t total, uint32_t na, VT *__restrict__ r, const VT *__restrict__ Mp, QmrDev q) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t c = e % na;
    const VT *tag = nullptr;
    r[e] = vsub(r[e], vmul(to_vt(q.alpha[c], tag), Mp[e]));
}

// d <- cd d + ca p;  x += d;  s <- (1 - c^2) s + c^2 r
template <class VT>
__global__ void k_qmr_dxs(uint32_t total, uint32_t na, VT *__restrict__ d, const VT *__restrict__ p,
                          double2 *__restrict__ x, VT *__restrict__ sres, const VT *__restrict__ r, QmrDev q) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t c = e % na;
    if (q.done[c]) return;
    const VT *tag = nullptr;
    const VT dv = vadd(vmul(to_vt(q.cd[c], tag), d[e]), vmul(to_vt(q.ca[c], tag), p[e]));
    d[e] = dv;
    x[e] = cadd(x[e], ld2(&dv));
    const double c2 = q.c2[c];
    const VT a = to_vt(make_double2(1.0 - c2, 0.0), tag), b = to_vt(make_double2(c2, 0.0), tag);
    sres[e] = vadd(vmul(a, sres[e]), vmul(b, r[e]));
}

// p <- r + beta p;  Dp <- Dr + beta Dp
template <class VT>
__global__ void k_qmr_p(uint32_t total, uint32_t na, VT *__restrict__ p, VT *__restrict__ Dp, const VT *__restrict__ r,
                        const VT *__restrict__ Dr, QmrDev q) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const uint32_t c = e % na;
    const VT *tag = nullptr;
    const VT b = to_vt(q.beta[c], tag);
    p[e] = vadd(r[e], vmul(b, p[e]));
    Dp[e] = vadd(Dr[e], vmul(b, Dp[e]));
}

// restart: r = p = s = FP64 residual, d = 0, xd = 0
template <class VT>
__global__ void k_qmr_restart_vec(uint32_t total, const double2 *__restrict__ r64, VT *__restrict__ r,
                                  VT *__restrict__ p, VT *__restrict__ sres, VT *__restrict__ d,
                                  double2 *__restrict__ xd) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const double2 v = r64[e];
    st2(r + e, v);
    st2(p + e, v);
    st2(sres + e, v);
    st2(d + e, czero());
    xd[e] = czero();
}

__global__ void k_qmr_restart_cols(int64_t na, const double2 *__restrict__ rnorm, const double *__restrict__ bnorm_a,
                                   double tol, double inner_red, QmrDev q) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= na) return;
    const double rn = rnorm[c].x;
    q.done[c] = (rn == 0.0) ? 1 : 0;
    q.breakdown[c] = 0;
    q.iters[c] = 0;
    q.tau[c] = rn;
    q.theta_old[c] = 0.0;
    q.target[c] = fmax(0.5 * tol * bnorm_a[c], inner_red * rn);
}

template <class VT>
static int qmr_impl(wfq_geom *g, const SolveArgs &a, cudaStream_t s, GmresOut *out) {
    Common cm;
    WFQ_TRY(cm.init(g, a, s));
    const int64_t n = cm.n, cc = cm.cc;
    const bool mixed = (a.prec == WFQ_PREC_MIXED);
    cm.residual_df = mixed;
    wfq_ctx *ctx = g->ctx;
    DevBuf<VT> r, p, Dp, Dr, Mp, sres, d;
    DevBuf<double2> rho, sigma, alpha, beta, cd, ca, xd;
    DevBuf<double> tau, theta, c2, target;
    DevBuf<int> done, iters, brk;
    DevBuf<unsigned char> scratch;
    for (DevBuf<VT> *b : {&r, &p, &Dp, &Dr, &Mp, &sres, &d}) WFQ_TRY(b->alloc(ctx, n * cc, s));
    for (DevBuf<double2> *b : {&rho, &sigma, &alpha, &beta, &cd, &ca}) WFQ_TRY(b->alloc(ctx, cc, s));
    WFQ_TRY(xd.alloc(ctx, n * cc, s));
    for (DevBuf<double> *b : {&tau, &theta, &c2, &target}) WFQ_TRY(b->alloc(ctx, cc, s));
    for (DevBuf<int> *b : {&done, &iters, &brk}) WFQ_TRY(b->alloc(ctx, cc, s));
    if (mixed) WFQ_TRY(scratch.alloc(ctx, mixed_scratch_bytes(g, cc), s));
    if (!a.warm) WFQ_CUDA(cudaMemsetAsync(a.q, 0, sizeof(double2) * n * cc, s));
    const double inner_red = mixed ? 1e-6 : 0.0;

    std::vector<int> act(cc), still, iters_h(cc, 0), brk_h(cc, 0), done_h, tmp_i, b_a;
    for (int64_t c = 0; c < cc; ++c) act[c] = (int)c;
    int total = 0, cycles = 0;
    WFQ_TRY(cm.select(act));
    WFQ_CUDA(cudaMemcpyAsync(cm.ra.ptr, cm.Ba.ptr, sizeof(double2) * n * cc, cudaMemcpyDeviceToDevice, s));
    WFQ_TRY(cm.colnorm(cm.ra.ptr, cc, cm.rnorm.ptr));
    // mixed: restart at the latest after this many iterations, so that the stagnation test
    // below sees every column regularly
    const int cycle_cap = mixed ? (a.refine_every > 0 ? a.refine_every : 300) : INT32_MAX;
    std::vector<double> prev_exact(cc, -1.0);
    std::vector<int> flat(cc, 0), slow_runs(cc, 0), esc;
    std::vector<char> inner_done(cc, 0);   // mixed: the column converged in the last inner run
    for (;;) {
        WFQ_TRY(cm.classify(act, a.rel_tol, still));
        // columns whose QMR broke down leave the active set; a mixed solve hands them, and
        // the columns that stalled over two restarts, to FP64 GMRES afterwards
        std::vector<int> keep;
        const size_t esc0 = esc.size();
        bool tighten = false;
        for (int c : still) {
            if (mixed && out) {
                const bool slow = prev_exact[c] >= 0.0 && cm.res_h[c] > STAGNATION_RATIO * prev_exact[c];
                flat[c] = slow && inner_done[c] ? flat[c] + 1 : 0;
                slow_runs[c] = slow ? slow_runs[c] + 1 : 0;
                prev_exact[c] = cm.res_h[c];
                if (flat[c] >= STAGNATION_CYCLES && !brk_h[c] && cm.can_tighten_residual()) tighten = true;
                if (brk_h[c] || flat[c] >= STAGNATION_CYCLES || slow_runs[c] >= SLOW_CYCLES) {
                    esc.push_back(c);
                    continue;
                }
            }
            if (!brk_h[c]) keep.push_back(c);
        }
        if (tighten) {
            // the floor is the residual's: recompute it with D in FP64 and carry on in mixed
            // precision (the classification below this `continue` escalates the columns whose
            // QMR broke down again, so none stays listed twice)
            esc.resize(esc0);
            cm.residual_exact = true;
            std::fill(flat.begin(), flat.end(), 0);
            std::fill(slow_runs.begin(), slow_runs.end(), 0);
            std::fill(prev_exact.begin(), prev_exact.end(), -1.0);
            trace("qmr mixed restart %d: residual floor of the regenerated double-float D; residuals from D in "
                  "FP64 from here", cycles);
            WFQ_TRY(cm.true_residual(a.q, (int64_t)act.size()));
            continue;
        }
        if (trace_on()) {
            double worst = 0.0;
            for (int c : act) worst = std::max(worst, cm.res_h[c]);
            trace("qmr %s restart %d: %zu of %zu columns active, %zu escalated, %d steps, max true rel. residual "
                  "%.3e", mixed ? "mixed" : "fp64", cycles, keep.size(), act.size(), esc.size(), total, worst);
        }
        if (keep.empty() || total >= a.max_iter) break;
        if (keep.size() != act.size()) WFQ_TRY(cm.narrow(act, keep));
        const int64_t na = (int64_t)act.size();
        // ---- one QMR run from the FP64 residual on the na active columns
        const uint32_t tot = (uint32_t)(n * na);
        QmrDev q{na, rho.ptr, sigma.ptr, alpha.ptr, beta.ptr, tau.ptr, theta.ptr, c2.ptr,
                 cd.ptr, ca.ptr, target.ptr, done.ptr, iters.ptr, brk.ptr};
        const RowSplit rs = row_split(n, na, cm.num_sms);
        const dim3 g1 = colpart_grid(rs.nrb, 1, na, rs.cx);
        const unsigned gw = nblocks(na * 32);
        auto dmul = [&](const VT *v, VT *u) -> int {
            if (mixed)
                return d_apply_mixed(g, na, reinterpret_cast<const float2 *>(v), reinterpret_cast<float2 *>(u),
                                     scratch.ptr, s);
            return solver_fp64_product(g, na, reinterpret_cast<const double2 *>(v), reinterpret_cast<double2 *>(u), s);
        };
        auto sparse = [&](const VT *u, const VT *x, VT *yv) -> int {
            if (mixed)
                return sparse_shift_fp32(g, na, reinterpret_cast<const float2 *>(u),
                                         reinterpret_cast<const float2 *>(x), cm.za.ptr,
                                         reinterpret_cast<float2 *>(yv), s);
            return sparse_shift_fp64(g, na, reinterpret_cast<const double2 *>(u),
                                     reinterpret_cast<const double2 *>(x), cm.za.ptr, reinterpret_cast<double2 *>(yv),
                                     s);
        };
        k_qmr_restart_cols<<<nblocks(na), 256, 0, s>>>(na, cm.rnorm.ptr, cm.bnorm_a.ptr, a.rel_tol, inner_red, q); note_launch();
        k_qmr_restart_vec<VT><<<nblocks(tot), 256, 0, s>>>(tot, cm.ra.ptr, r.ptr, p.ptr, sres.ptr, d.ptr, xd.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        WFQ_TRY(dmul(r.ptr, Dr.ptr));
        WFQ_CUDA(cudaMemcpyAsync(Dp.ptr, Dr.ptr, sizeof(VT) * n * na, cudaMemcpyDeviceToDevice, s));
        k_colpart<VT><<<g1, 256, 0, s>>>(n, na, 1, RED_BILIN, r.ptr, 0, Dr.ptr, rs.cx, rs.ry, rs.nrb, cm.partial.ptr); note_launch();
        k_qmr_fin<<<gw, 256, 0, s>>>(na, rs.nrb, QF_START, cm.partial.ptr, q); note_launch();
        int since = 0;
        done_h.assign(na, 0);
        for (;;) {
            if (total >= a.max_iter) break;
            WFQ_TRY(sparse(Dp.ptr, p.ptr, Mp.ptr));  // M p = (Kbar - P) D p - z p
            k_colpart<VT><<<g1, 256, 0, s>>>(n, na, 1, RED_BILIN, Dp.ptr, 0, Mp.ptr, rs.cx, rs.ry, rs.nrb, cm.partial.ptr); note_launch();
            k_qmr_fin<<<gw, 256, 0, s>>>(na, rs.nrb, QF_SIGMA, cm.partial.ptr, q); note_launch();
            k_qmr_r<VT><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, r.ptr, Mp.ptr, q); note_launch();
            k_colpart<VT><<<g1, 256, 0, s>>>(n, na, 1, RED_NORM2, nullptr, 0, r.ptr, rs.cx, rs.ry, rs.nrb, cm.partial.ptr); note_launch();
            k_qmr_fin<<<gw, 256, 0, s>>>(na, rs.nrb, QF_RNORM, cm.partial.ptr, q); note_launch();
            k_qmr_dxs<VT><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, d.ptr, p.ptr, xd.ptr, sres.ptr, r.ptr, q); note_launch();
            k_colpart<VT><<<g1, 256, 0, s>>>(n, na, 1, RED_NORM2, nullptr, 0, sres.ptr, rs.cx, rs.ry, rs.nrb, cm.partial.ptr); note_launch();
            k_qmr_fin<<<gw, 256, 0, s>>>(na, rs.nrb, QF_SNORM, cm.partial.ptr, q); note_launch();
            WFQ_CUDA(cudaGetLastError());
            ++total;
            ++since;
            WFQ_CUDA(cudaMemcpyAsync(done_h.data(), done.ptr, sizeof(int) * na, cudaMemcpyDeviceToHost, s));
            WFQ_CUDA(cudaStreamSynchronize(s));
            if (std::all_of(done_h.begin(), done_h.end(), [](int v) { return v != 0; })) break;
            if (since >= cycle_cap) break;
            WFQ_TRY(dmul(r.ptr, Dr.ptr));   // the one D product of the iteration
            k_colpart<VT><<<g1, 256, 0, s>>>(n, na, 1, RED_BILIN, r.ptr, 0, Dr.ptr, rs.cx, rs.ry, rs.nrb, cm.partial.ptr); note_launch();
            k_qmr_fin<<<gw, 256, 0, s>>>(na, rs.nrb, QF_RHO, cm.partial.ptr, q); note_launch();
            k_qmr_p<VT><<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, p.ptr, Dp.ptr, r.ptr, Dr.ptr, q); note_launch();
            WFQ_CUDA(cudaGetLastError());
        }
        k_scatter_add<<<nblocks(tot), 256, 0, s>>>(tot, (uint32_t)na, cc, cm.idx.ptr, xd.ptr, a.q); note_launch();
        tmp_i.assign(na, 0);
        b_a.assign(na, 0);
        WFQ_CUDA(cudaMemcpyAsync(tmp_i.data(), iters.ptr, sizeof(int) * na, cudaMemcpyDeviceToHost, s));
        WFQ_CUDA(cudaMemcpyAsync(b_a.data(), brk.ptr, sizeof(int) * na, cudaMemcpyDeviceToHost, s));
        WFQ_CUDA(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < na; ++k) {
            iters_h[act[k]] += tmp_i[k];
            if (b_a[k]) brk_h[act[k]] = 1;
            inner_done[act[k]] = done_h[k] != 0;
        }
        ++cycles;
        WFQ_TRY(cm.true_residual(a.q, na));
    }
    if (out) {
        std::sort(esc.begin(), esc.end());
        out->escalate = esc;
        out->res = cm.res_h;
        out->iters = iters_h;
        out->cycles = cycles;
    }
    return finish_stats(a, cm, iters_h, cycles, brk_h);
}

int solve_qmr(wfq_geom *g, const SolveArgs &a, cudaStream_t s) {
    if (a.prec != WFQ_PREC_MIXED) return qmr_impl<double2>(g, a, s, nullptr);
    GmresOut o1;
    const int rc = qmr_impl<float2>(g, a, s, &o1);
    if (o1.escalate.empty() || (rc != WFQ_OK && rc != WFQ_ENOCONV && rc != WFQ_EBREAKDOWN)) return rc;
    return continue_columns(g, a, o1.escalate, o1.res, o1.iters, WFQ_PREC_FP64, 50, s);
}

}  // namespace wfq
