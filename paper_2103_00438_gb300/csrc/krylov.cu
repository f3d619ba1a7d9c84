// Krylov shells of Section 3 on the GPU, batched over independent complex columns
// (one column per (frequency, field direction); all columns share D and Kbar):
//   - GMRES / GMRES(m) (Eq. 24): Arnoldi with modified Gram-Schmidt, Givens QR of the
//     Hessenberg matrix, x = x0 + V y.  Inner products, norms, Givens rotations and
//     the solution update are FP64; the basis is complex128 (FP64 operator) or
//     complex64 (mixed operator).  Every restart cycle starts from the FP64 true
//     residual r = R - (A - zI) x, which makes the mixed form an iterative refinement.
//   - J-symmetric QMR from BCG without look-ahead (J = D, Eq. 18): BCG with the shadow
//     vectors J r and J p, smoothed into the QMR iterate.  The D p needed for A p comes
//     from the recurrence D p <- D r + beta D p, so each iteration needs one D product
//     (D r), which also gives the bilinear form r^T D r.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"

namespace wfq {

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

// ------------------------------------------------------------------ column reductions

// Launch geometry of the column-wise kernels: 256 threads; CX lanes across columns
// (power of two, <= 32), RY = 256 / CX rows in flight; each block owns a contiguous
// chunk of atom rows.  Partial sums per (block, column) are reduced in block order by
// the last block to finish (deterministic, independent of scheduling).
struct ColGrid {
    int cx = 32, ry = 8, nblk = 1;
};

static ColGrid col_grid(int64_t n, int64_t cc, int num_sms) {
    ColGrid g;
    int cx = 1;
    while (cx < cc && cx < 32) cx <<= 1;
    g.cx = cx;
    g.ry = 256 / cx;
    int64_t want = std::max<int64_t>(1, (n + 63) / 64);
    g.nblk = (int)std::min<int64_t>(want, (int64_t)2 * std::max(1, num_sms));
    return g;
}

struct Red {
    double2 *partial;   // nblk * cc
    unsigned *ticket;   // one counter, zero between launches
};

// Block-level reduction over ty for each tx; writes partial[block][c].
__device__ __forceinline__ void block_partial(double2 acc, int cx, int ry, int tx, int ty, int64_t c,
                                              int64_t cc, double2 *sm, double2 *partial) {
    sm[ty * cx + tx] = acc;
    __syncthreads();
    for (int s = ry >> 1; s > 0; s >>= 1) {
        if (ty < s) sm[ty * cx + tx] = cadd(sm[ty * cx + tx], sm[(ty + s) * cx + tx]);
        __syncthreads();
    }
    if (ty == 0 && c < cc) partial[(int64_t)blockIdx.x * cc + c] = sm[tx];
    __syncthreads();
}

// Returns true in the block that finished last (after every block wrote its partials).
__device__ __forceinline__ bool last_block(unsigned *ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        if (threadIdx.x == 0) *ticket = 0u;
    }
    return is_last;
}

__device__ __forceinline__ double2 sum_partials(const double2 *partial, int nblk, int64_t cc, int64_t c) {
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nblk; ++b) s = cadd(s, __ldcg(partial + (int64_t)b * cc + c));
    return s;
}

// ------------------------------------------------------------------ GMRES state

struct GmresDev {
    int m;
    int64_t cc;
    double2 *H;      // [(m+1) * m][cc]: H(i, j) of column c at (i * m + j) * cc + c
    double *cs;      // [m][cc]
    double2 *sn;     // [m][cc]
    double2 *g;      // [m+1][cc]
    double *target;  // [cc] absolute residual-estimate target of this cycle
    int *done;       // [cc]
    int *jdone;      // [cc] Arnoldi steps used by the column in this cycle
    int *iters;      // [cc] total Krylov iterations
};

// Givens QR update of column j of H for column c (complex rotations with real cosine).
__device__ void givens_step(const GmresDev &st, int64_t c, int j) {
    if (st.done[c]) return;
    const int m = st.m;
    const int64_t cc = st.cc;
    auto Hp = [&](int i, int jj) { return st.H + ((int64_t)i * m + jj) * cc + c; };
    for (int i = 0; i < j; ++i) {
        double cs = st.cs[(int64_t)i * cc + c];
        double2 sn = st.sn[(int64_t)i * cc + c];
        double2 a = *Hp(i, j), b = *Hp(i + 1, j);
        *Hp(i, j) = cadd(cscale(cs, a), cmul(sn, b));
        *Hp(i + 1, j) = csub(cscale(cs, b), cjmul(sn, a));
    }
    double2 a = *Hp(j, j);
    double hb = Hp(j + 1, j)->x;  // real, >= 0 (a norm)
    double na = sqrt(cabs2(a));
    double nu = sqrt(na * na + hb * hb);
    double cs;
    double2 sn, rdiag;
    if (nu == 0.0) {
        cs = 1.0;
        sn = make_double2(0.0, 0.0);
        rdiag = a;
    } else if (na == 0.0) {
        cs = 0.0;
        sn = make_double2(1.0, 0.0);
        rdiag = make_double2(hb, 0.0);
    } else {
        double2 ph = cscale(1.0 / na, a);
        cs = na / nu;
        sn = cscale(hb / nu, ph);
        rdiag = cscale(nu, ph);
    }
    st.cs[(int64_t)j * cc + c] = cs;
    st.sn[(int64_t)j * cc + c] = sn;
    *Hp(j, j) = rdiag;
    *Hp(j + 1, j) = make_double2(0.0, 0.0);
    double2 gj = st.g[(int64_t)j * cc + c];
    st.g[(int64_t)(j + 1) * cc + c] = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
    st.g[(int64_t)j * cc + c] = cscale(cs, gj);
    st.iters[c] += 1;
    double res = sqrt(cabs2(st.g[(int64_t)(j + 1) * cc + c]));
    if (res <= st.target[c] || hb == 0.0 || nu == 0.0) {
        st.done[c] = 1;
        st.jdone[c] = j + 1;
    }
}

enum { MODE_DOT = 0, MODE_NORM = 1, MODE_NORM_GIVENS = 2 };

// One modified Gram-Schmidt step on w (columnwise):
//   if hprev: w <- w - hprev[c] * vprev            (finishes the previous projection)
//   MODE_DOT:  out[c] = <vi, w>  (conjugated)
//   MODE_NORM: out[c] = ||w||   (stored in .x);  MODE_NORM_GIVENS also runs givens_step
template <class VT>
__global__ void __launch_bounds__(256) k_mgs(int64_t n, int64_t cc, int cx, int ry, int mode, VT *__restrict__ w,
                                             const VT *__restrict__ vprev, const double2 *__restrict__ hprev,
                                             const VT *__restrict__ vi, Red red, double2 *__restrict__ out,
                                             GmresDev st, int j) {
    __shared__ double2 sm[256];
    const int tx = threadIdx.x % cx, ty = threadIdx.x / cx;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    for (int64_t c0 = 0; c0 < cc; c0 += cx) {
        const int64_t c = c0 + tx;
        double2 acc = make_double2(0.0, 0.0);
        if (c < cc) {
            double2 hp = hprev ? hprev[c] : make_double2(0.0, 0.0);
            for (int64_t r = r0 + ty; r < r1; r += ry) {
                const int64_t e = r * cc + c;
                double2 wv = ld2(w + e);
                if (hprev) {
                    wv = csub(wv, cmul(hp, ld2(vprev + e)));
                    st2(w + e, wv);
                    wv = ld2(w + e);   // continue with the stored (rounded) value
                }
                if (mode == MODE_DOT)
                    acc = cadd(acc, cjmul(ld2(vi + e), wv));
                else
                    acc.x += cabs2(wv);
            }
        }
        block_partial(acc, cx, ry, tx, ty, c, cc, sm, red.partial);
    }
    if (!last_block(red.ticket)) return;
    for (int64_t c = threadIdx.x; c < cc; c += blockDim.x) {
        double2 s = sum_partials(red.partial, gridDim.x, cc, c);
        if (mode == MODE_DOT) {
            out[c] = s;
        } else {
            // MODE_NORM_GIVENS: out is the per-column norm buffer read by k_scale; H(j+1, j)
            // gets the same value and is then rotated to zero by the Givens step.
            out[c] = make_double2(sqrt(s.x), 0.0);
            if (mode == MODE_NORM_GIVENS) {
                st.H[((int64_t)(j + 1) * st.m + j) * cc + c] = out[c];
                givens_step(st, c, j);
            }
        }
    }
}

// v <- v / h (h = H(j+1, j)); zero for columns that are done (their later basis vectors
// are not used and must stay finite).
template <class VT>
__global__ void k_scale(int64_t n, int64_t cc, VT *__restrict__ v, const double2 *__restrict__ h,
                        const int *__restrict__ done) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * cc) return;
    int64_t c = e % cc;
    double hv = h[c].x;
    double s = (done[c] || hv == 0.0) ? 0.0 : 1.0 / hv;
    st2(v + e, cscale(s, ld2(v + e)));
}

// r = B - Y (FP64)
__global__ void k_residual(int64_t total, const double2 *__restrict__ B, const double2 *__restrict__ Y,
                           double2 *__restrict__ r) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < total) r[e] = csub(B[e], Y[e]);
}

// B[i][f*ndir + d] = R[i][d]
__global__ void k_make_b(int64_t n, int64_t nfreq, int ndir, const double *__restrict__ R,
                         double2 *__restrict__ B) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t cc = nfreq * ndir;
    if (e >= n * cc) return;
    int64_t i = e / cc, c = e % cc;
    B[e] = make_double2(R[i * ndir + (int)(c % ndir)], 0.0);
}

// Per-column set-up of a cycle from the FP64 residual norms.
__global__ void k_cycle_cols(int64_t cc, const double2 *__restrict__ rnorm, const double2 *__restrict__ bnorm,
                             double tol, double inner_red, GmresDev st, int *__restrict__ converged) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cc) return;
    double rn = rnorm[c].x, bn = bnorm[c].x;
    int conv = (rn <= tol * bn) ? 1 : 0;
    converged[c] = conv;
    st.done[c] = (conv || rn == 0.0) ? 1 : 0;
    st.jdone[c] = 0;
    st.g[c] = make_double2(rn, 0.0);
    st.target[c] = fmax(0.5 * tol * bn, inner_red * rn);
}

// v0 = r / ||r|| (zero for done columns)
template <class VT>
__global__ void k_start_basis(int64_t n, int64_t cc, const double2 *__restrict__ r, const double2 *__restrict__ rnorm,
                              const int *__restrict__ done, VT *__restrict__ v0) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * cc) return;
    int64_t c = e % cc;
    double s = (done[c] || rnorm[c].x == 0.0) ? 0.0 : 1.0 / rnorm[c].x;
    st2(v0 + e, cscale(s, r[e]));
}

// y = R^{-1} g on the first jd rows (R = rotated H), one thread per column.
__global__ void k_backsolve(int64_t cc, int jlast, GmresDev st, double2 *__restrict__ y) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cc) return;
    const int m = st.m;
    int jd = st.done[c] ? st.jdone[c] : (jlast + 1);
    st.jdone[c] = jd;
    for (int l = jd - 1; l >= 0; --l) {
        double2 s = st.g[(int64_t)l * cc + c];
        for (int k = l + 1; k < jd; ++k)
            s = csub(s, cmul(st.H[((int64_t)l * m + k) * cc + c], y[(int64_t)k * cc + c]));
        y[(int64_t)l * cc + c] = cdiv(s, st.H[((int64_t)l * m + l) * cc + c]);
    }
}

// x += sum_{l < jd_c} y_l V_l
template <class VT>
__global__ void k_update_x(int64_t n, int64_t cc, int jmax, const VT *__restrict__ V, const double2 *__restrict__ y,
                           const int *__restrict__ jdone, double2 *__restrict__ x) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * cc) return;
    int64_t c = e % cc;
    int jd = jdone[c];
    double2 s = x[e];
    const int64_t stride = n * cc;
    for (int l = 0; l < jmax && l < jd; ++l) s = cadd(s, cmul(y[(int64_t)l * cc + c], ld2(V + l * stride + e)));
    x[e] = s;
}

__global__ void k_set_z(int64_t nfreq, int ndir, const double *__restrict__ omega, double n0, double tau,
                        double2 *__restrict__ z) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nfreq * ndir) return;
    double w = omega[c / ndir];
    double f = -w / (2.0 * n0 * tau);
    z[c] = make_double2(f * w * tau, f);
}

static inline unsigned nblocks(int64_t total, int t = 256) { return (unsigned)((total + t - 1) / t); }

// ------------------------------------------------------------------ shared solver set-up

struct Common {
    wfq_geom *g;
    cudaStream_t s;
    int64_t n, cc;
    ColGrid cg;
    DevBuf<double2> B, r, Y64, U64, z, partial, bnorm, rnorm, tmp;
    DevBuf<double> R, dirs, omega;
    DevBuf<unsigned> ticket;
    DevBuf<int> converged;
    Red red;

    int init(wfq_geom *geom, const SolveArgs &a, cudaStream_t stream) {
        g = geom;
        s = stream;
        n = g->n;
        cc = a.nfreq * a.ndir;
        cg = col_grid(n, cc, g->ctx->num_sms);
        wfq_ctx *ctx = g->ctx;
        WFQ_TRY(B.alloc(ctx, n * cc, s));
        WFQ_TRY(r.alloc(ctx, n * cc, s));
        WFQ_TRY(Y64.alloc(ctx, n * cc, s));
        WFQ_TRY(U64.alloc(ctx, n * cc, s));
        WFQ_TRY(z.alloc(ctx, cc, s));
        WFQ_TRY(partial.alloc(ctx, (size_t)cg.nblk * cc, s));
        WFQ_TRY(bnorm.alloc(ctx, cc, s));
        WFQ_TRY(rnorm.alloc(ctx, cc, s));
        WFQ_TRY(tmp.alloc(ctx, cc, s));
        WFQ_TRY(R.alloc(ctx, n * a.ndir, s));
        WFQ_TRY(dirs.alloc(ctx, 3 * a.ndir, s));
        WFQ_TRY(omega.alloc(ctx, a.nfreq, s));
        WFQ_TRY(ticket.alloc(ctx, 1, s));
        WFQ_TRY(converged.alloc(ctx, cc, s));
        WFQ_CUDA(cudaMemsetAsync(ticket.ptr, 0, sizeof(unsigned), s));
        WFQ_CUDA(cudaMemcpyAsync(dirs.ptr, a.dirs, sizeof(double) * 3 * a.ndir, cudaMemcpyHostToDevice, s));
        WFQ_CUDA(cudaMemcpyAsync(omega.ptr, a.omega, sizeof(double) * a.nfreq, cudaMemcpyHostToDevice, s));
        red.partial = partial.ptr;
        red.ticket = ticket.ptr;
        k_set_z<<<nblocks(cc), 256, 0, s>>>(a.nfreq, a.ndir, omega.ptr, g->p.n0, g->p.tau, z.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        WFQ_TRY(launch_rhs(g, a.ndir, dirs.ptr, a.E0, R.ptr, s));
        k_make_b<<<nblocks(n * cc), 256, 0, s>>>(n, a.nfreq, a.ndir, R.ptr, B.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        WFQ_TRY(colnorm(B.ptr, bnorm.ptr));
        return WFQ_OK;
    }

    // out[c].x = ||v_c||
    int colnorm(double2 *v, double2 *out) {
        GmresDev dummy{};
        k_mgs<double2><<<cg.nblk, 256, 0, s>>>(n, cc, cg.cx, cg.ry, MODE_NORM, v, nullptr, nullptr, nullptr, red,
                                               out, dummy, 0); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }

    // Y64 = (A - zI) x in FP64; r = B - Y64; rnorm = ||r||
    int true_residual(const double2 *x) {
        WFQ_TRY(d_apply_fp64(g, cc, x, U64.ptr, s));
        WFQ_TRY(sparse_shift_fp64(g, cc, U64.ptr, x, z.ptr, Y64.ptr, s));
        k_residual<<<nblocks(n * cc), 256, 0, s>>>(n * cc, B.ptr, Y64.ptr, r.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return colnorm(r.ptr, rnorm.ptr);
    }
};

static int fill_stats(const SolveArgs &a, Common &cm, const std::vector<int> &iters, int cycles, int status,
                      bool breakdown_any, const std::vector<int> &breakdown) {
    WFQ_TRY(check_device_error(cm.g->ctx, cm.s));
    std::vector<double2> rn(cm.cc), bn(cm.cc);
    WFQ_CUDA(cudaMemcpyAsync(rn.data(), cm.rnorm.ptr, sizeof(double2) * cm.cc, cudaMemcpyDeviceToHost, cm.s));
    WFQ_CUDA(cudaMemcpyAsync(bn.data(), cm.bnorm.ptr, sizeof(double2) * cm.cc, cudaMemcpyDeviceToHost, cm.s));
    WFQ_CUDA(cudaStreamSynchronize(cm.s));
    bool all = true;
    for (int64_t c = 0; c < cm.cc; ++c) {
        double rel = bn[c].x > 0 ? rn[c].x / bn[c].x : 0.0;
        bool ok = rel <= a.rel_tol;
        all = all && ok;
        if (a.stats) {
            wfq_stats &st = a.stats[c];
            st.iters = iters.empty() ? 0 : iters[c];
            st.restarts = std::max(0, cycles - 1);
            st.refinements = (a.prec == WFQ_PREC_MIXED) ? std::max(0, cycles - 1) : 0;
            st.rel_residual = rel;
            st.rmse = rn[c].x / std::sqrt((double)cm.n);
            st.status = ok ? WFQ_OK : ((breakdown_any && !breakdown.empty() && breakdown[c]) ? WFQ_EBREAKDOWN : WFQ_ENOCONV);
        }
    }
    (void)status;
    if (all) return WFQ_OK;
    if (breakdown_any) return fail(WFQ_EBREAKDOWN, "QMR breakdown (rho or sigma = 0) without convergence");
    return fail(WFQ_ENOCONV, "iteration limit reached before rel_tol in some column");
}

// ------------------------------------------------------------------ GMRES

template <class VT>
static int gmres_impl(wfq_geom *g, const SolveArgs &a, cudaStream_t s) {
    Common cm;
    WFQ_TRY(cm.init(g, a, s));
    const int64_t n = cm.n, cc = cm.cc, nc = n * cc;
    const bool mixed = (a.prec == WFQ_PREC_MIXED);
    int m = a.m > 0 ? std::min(a.m, a.max_iter) : a.max_iter;
    m = std::max(1, m);
    wfq_ctx *ctx = g->ctx;

    DevBuf<VT> V;
    DevBuf<double2> H, sn, gv, y;
    DevBuf<double> cs, target;
    DevBuf<int> done, jdone, iters;
    DevBuf<float2> U32;
    DevBuf<unsigned char> scratch;
    WFQ_TRY(V.alloc(ctx, (size_t)(m + 1) * nc, s));
    WFQ_TRY(H.alloc(ctx, (size_t)(m + 1) * m * cc, s));
    WFQ_TRY(sn.alloc(ctx, (size_t)m * cc, s));
    WFQ_TRY(gv.alloc(ctx, (size_t)(m + 1) * cc, s));
    WFQ_TRY(y.alloc(ctx, (size_t)m * cc, s));
    WFQ_TRY(cs.alloc(ctx, (size_t)m * cc, s));
    WFQ_TRY(target.alloc(ctx, cc, s));
    WFQ_TRY(done.alloc(ctx, cc, s));
    WFQ_TRY(jdone.alloc(ctx, cc, s));
    WFQ_TRY(iters.alloc(ctx, cc, s));
    if (mixed) {
        WFQ_TRY(U32.alloc(ctx, nc, s));
        WFQ_TRY(scratch.alloc(ctx, mixed_scratch_bytes(g, cc), s));
    }
    WFQ_CUDA(cudaMemsetAsync(iters.ptr, 0, sizeof(int) * cc, s));
    WFQ_CUDA(cudaMemsetAsync(H.ptr, 0, sizeof(double2) * (m + 1) * m * cc, s));
    WFQ_CUDA(cudaMemsetAsync(a.q, 0, sizeof(double2) * nc, s));

    GmresDev st{m, cc, H.ptr, cs.ptr, sn.ptr, gv.ptr, target.ptr, done.ptr, jdone.ptr, iters.ptr};
    const double inner_red = mixed ? 1e-6 : 0.0;
    std::vector<int> done_h(cc), conv_h(cc);
    int total = 0, cycles = 0;
    const ColGrid cg = cm.cg;

    for (;;) {
        if (cycles == 0) {
            WFQ_CUDA(cudaMemcpyAsync(cm.r.ptr, cm.B.ptr, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
            WFQ_CUDA(cudaMemcpyAsync(cm.rnorm.ptr, cm.bnorm.ptr, sizeof(double2) * cc, cudaMemcpyDeviceToDevice, s));
        } else {
            WFQ_TRY(cm.true_residual(a.q));
        }
        k_cycle_cols<<<nblocks(cc), 256, 0, s>>>(cc, cm.rnorm.ptr, cm.bnorm.ptr, a.rel_tol, inner_red, st,
                                                 cm.converged.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        WFQ_CUDA(cudaMemcpyAsync(conv_h.data(), cm.converged.ptr, sizeof(int) * cc, cudaMemcpyDeviceToHost, s));
        WFQ_TRY(check_device_error(g->ctx, s));
        bool all_conv = std::all_of(conv_h.begin(), conv_h.end(), [](int v) { return v != 0; });
        if (all_conv || total >= a.max_iter) break;

        k_start_basis<VT><<<nblocks(nc), 256, 0, s>>>(n, cc, cm.r.ptr, cm.rnorm.ptr, done.ptr, V.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        int jlast = -1;
        for (int j = 0; j < m && total < a.max_iter; ++j) {
            VT *vj = V.ptr + (int64_t)j * nc;
            VT *w = V.ptr + (int64_t)(j + 1) * nc;
            if (mixed) {
                WFQ_TRY(d_apply_mixed(g, cc, reinterpret_cast<const float2 *>(vj), U32.ptr, scratch.ptr, s));
                WFQ_TRY(sparse_shift_fp32(g, cc, U32.ptr, reinterpret_cast<const float2 *>(vj), cm.z.ptr,
                                          reinterpret_cast<float2 *>(w), s));
            } else {
                WFQ_TRY(d_apply_fp64(g, cc, reinterpret_cast<const double2 *>(vj), cm.U64.ptr, s));
                WFQ_TRY(sparse_shift_fp64(g, cc, cm.U64.ptr, reinterpret_cast<const double2 *>(vj), cm.z.ptr,
                                          reinterpret_cast<double2 *>(w), s));
            }
            // modified Gram-Schmidt: step i projects out v_i after removing v_{i-1}
            for (int i = 0; i <= j; ++i) {
                const double2 *hprev = i > 0 ? H.ptr + ((int64_t)(i - 1) * m + j) * cc : nullptr;
                const VT *vprev = i > 0 ? V.ptr + (int64_t)(i - 1) * nc : nullptr;
                k_mgs<VT><<<cg.nblk, 256, 0, s>>>(n, cc, cg.cx, cg.ry, MODE_DOT, w, vprev, hprev,
                                                  V.ptr + (int64_t)i * nc, cm.red,
                                                  H.ptr + ((int64_t)i * m + j) * cc, st, j); note_launch();
            }
            k_mgs<VT><<<cg.nblk, 256, 0, s>>>(n, cc, cg.cx, cg.ry, MODE_NORM_GIVENS, w, V.ptr + (int64_t)j * nc,
                                              H.ptr + ((int64_t)j * m + j) * cc, nullptr, cm.red, cm.tmp.ptr, st, j); note_launch();
            WFQ_CUDA(cudaGetLastError());
            k_scale<VT><<<nblocks(nc), 256, 0, s>>>(n, cc, w, cm.tmp.ptr, done.ptr); note_launch();
            WFQ_CUDA(cudaGetLastError());
            ++total;
            jlast = j;
            WFQ_CUDA(cudaMemcpyAsync(done_h.data(), done.ptr, sizeof(int) * cc, cudaMemcpyDeviceToHost, s));
            WFQ_CUDA(cudaStreamSynchronize(s));
            if (std::all_of(done_h.begin(), done_h.end(), [](int v) { return v != 0; })) break;
        }
        if (jlast >= 0) {
            k_backsolve<<<nblocks(cc), 256, 0, s>>>(cc, jlast, st, y.ptr); note_launch();
            WFQ_CUDA(cudaGetLastError());
            k_update_x<VT><<<nblocks(nc), 256, 0, s>>>(n, cc, jlast + 1, V.ptr, y.ptr, jdone.ptr, a.q); note_launch();
            WFQ_CUDA(cudaGetLastError());
        }
        ++cycles;
    }
    // final FP64 true residual for the statistics
    if (cycles > 0) WFQ_TRY(cm.true_residual(a.q));
    std::vector<int> it(cc);
    WFQ_CUDA(cudaMemcpyAsync(it.data(), iters.ptr, sizeof(int) * cc, cudaMemcpyDeviceToHost, s));
    return fill_stats(a, cm, it, cycles, 0, false, {});
}

int solve_gmres(wfq_geom *g, const SolveArgs &a, cudaStream_t s) {
    if (a.prec == WFQ_PREC_MIXED) return gmres_impl<float2>(g, a, s);
    return gmres_impl<double2>(g, a, s);
}

// ------------------------------------------------------------------ QMR

struct QmrDev {
    int64_t cc;
    double2 *rho, *sigma, *alpha, *beta;
    double *tau, *theta_old, *ca_c2;   // ca_c2: c^2 of the current step
    double2 *cd, *ca;                  // d <- cd d + ca p
    double *target;
    int *done, *iters, *breakdown;
};

// Bilinear column reduction sum_i a_i b_i (no conjugation) with an optional fused
// AXPY before it, and a per-column finalize.
enum { QF_SIGMA = 0, QF_RNORM = 1, QF_SNORM = 2, QF_RHO = 3, QF_RESTART = 4 };

template <class VT>
__global__ void __launch_bounds__(256) k_qmr_red(int64_t n, int64_t cc, int cx, int ry, int kind,
                                                 const VT *__restrict__ a, const VT *__restrict__ b, Red red,
                                                 QmrDev q) {
    __shared__ double2 sm[256];
    const int tx = threadIdx.x % cx, ty = threadIdx.x / cx;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    for (int64_t c0 = 0; c0 < cc; c0 += cx) {
        const int64_t c = c0 + tx;
        double2 acc = make_double2(0.0, 0.0);
        if (c < cc) {
            for (int64_t r = r0 + ty; r < r1; r += ry) {
                const int64_t e = r * cc + c;
                double2 av = ld2(a + e);
                if (kind == QF_SIGMA || kind == QF_RHO || kind == QF_RESTART)
                    acc = cadd(acc, cmul(av, ld2(b + e)));
                else
                    acc.x += cabs2(av);
            }
        }
        block_partial(acc, cx, ry, tx, ty, c, cc, sm, red.partial);
    }
    if (!last_block(red.ticket)) return;
    for (int64_t c = threadIdx.x; c < cc; c += blockDim.x) {
        double2 s = sum_partials(red.partial, gridDim.x, cc, c);
        const bool dn = q.done[c] != 0;
        if (kind == QF_SIGMA) {
            q.sigma[c] = s;
            if (dn) {
                q.alpha[c] = make_double2(0.0, 0.0);
            } else if (s.x == 0.0 && s.y == 0.0) {
                q.breakdown[c] = 1;
                q.done[c] = 1;
                q.alpha[c] = make_double2(0.0, 0.0);
            } else {
                q.alpha[c] = cdiv(q.rho[c], s);
            }
        } else if (kind == QF_RNORM) {
            // QMR smoothing weights from the BCG residual norm
            double rn = sqrt(s.x);
            if (dn) {
                q.cd[c] = make_double2(0.0, 0.0);
                q.ca[c] = make_double2(0.0, 0.0);
                q.ca_c2[c] = 0.0;
            } else {
                double th = rn / q.tau[c];
                double c2 = 1.0 / (1.0 + th * th);
                q.cd[c] = make_double2(c2 * q.theta_old[c] * q.theta_old[c], 0.0);
                q.ca[c] = cscale(c2, q.alpha[c]);
                q.ca_c2[c] = c2;
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
                q.beta[c] = make_double2(0.0, 0.0);
            } else if (s.x == 0.0 && s.y == 0.0) {
                q.breakdown[c] = 1;
                q.done[c] = 1;
                q.beta[c] = make_double2(0.0, 0.0);
            } else {
                q.beta[c] = cdiv(s, q.rho[c]);
                q.rho[c] = s;
            }
        } else {  // QF_RESTART: rho = r^T D r of the fresh residual
            q.rho[c] = s;
            if (!dn && s.x == 0.0 && s.y == 0.0) {
                q.breakdown[c] = 1;
                q.done[c] = 1;
            }
        }
    }
}

// r <- r - alpha Mp
template <class VT>
__global__ void k_qmr_r(int64_t total, int64_t cc, VT *__restrict__ r, const VT *__restrict__ Mp, QmrDev q) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int64_t c = e % cc;
    st2(r + e, csub(ld2(r + e), cmul(q.alpha[c], ld2(Mp + e))));
}

// d <- cd d + ca p;  x += d;  s <- (1 - c^2) s + c^2 r
template <class VT>
__global__ void k_qmr_dxs(int64_t total, int64_t cc, VT *__restrict__ d, const VT *__restrict__ p,
                          double2 *__restrict__ x, VT *__restrict__ sres, const VT *__restrict__ r, QmrDev q) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int64_t c = e % cc;
    if (q.done[c]) return;
    double2 dv = cadd(cmul(q.cd[c], ld2(d + e)), cmul(q.ca[c], ld2(p + e)));
    st2(d + e, dv);
    x[e] = cadd(x[e], dv);
    double c2 = q.ca_c2[c];
    st2(sres + e, cadd(cscale(1.0 - c2, ld2(sres + e)), cscale(c2, ld2(r + e))));
}

// p <- r + beta p;  Dp <- Dr + beta Dp
template <class VT>
__global__ void k_qmr_p(int64_t total, int64_t cc, VT *__restrict__ p, VT *__restrict__ Dp, const VT *__restrict__ r,
                        const VT *__restrict__ Dr, QmrDev q) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int64_t c = e % cc;
    double2 b = q.beta[c];
    st2(p + e, cadd(ld2(r + e), cmul(b, ld2(p + e))));
    st2(Dp + e, cadd(ld2(Dr + e), cmul(b, ld2(Dp + e))));
}

// restart: r, p, s from the FP64 residual (zero for converged columns); d = 0
template <class VT>
__global__ void k_qmr_restart_vec(int64_t total, int64_t cc, const double2 *__restrict__ r64,
                                  const int *__restrict__ conv, VT *__restrict__ r, VT *__restrict__ p,
                                  VT *__restrict__ sres, VT *__restrict__ d) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int64_t c = e % cc;
    double2 v = conv[c] ? make_double2(0.0, 0.0) : r64[e];
    st2(r + e, v);
    st2(p + e, v);
    st2(sres + e, v);
    st2(d + e, make_double2(0.0, 0.0));
}

__global__ void k_qmr_restart_cols(int64_t cc, const double2 *__restrict__ rnorm, const double2 *__restrict__ bnorm,
                                   double tol, double inner_red, QmrDev q, int *__restrict__ converged) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cc) return;
    double rn = rnorm[c].x, bn = bnorm[c].x;
    int conv = (rn <= tol * bn) ? 1 : 0;
    converged[c] = conv;
    q.done[c] = (conv || rn == 0.0) ? 1 : 0;
    q.tau[c] = rn;
    q.theta_old[c] = 0.0;
    q.target[c] = fmax(0.5 * tol * bn, inner_red * rn);
}

template <class VT>
static int qmr_impl(wfq_geom *g, const SolveArgs &a, cudaStream_t s) {
    Common cm;
    WFQ_TRY(cm.init(g, a, s));
    const int64_t n = cm.n, cc = cm.cc, nc = n * cc;
    const bool mixed = (a.prec == WFQ_PREC_MIXED);
    wfq_ctx *ctx = g->ctx;
    DevBuf<VT> r, p, Dp, Dr, Mp, sres, d;
    DevBuf<double2> rho, sigma, alpha, beta, cd, ca;
    DevBuf<double> tau, theta, c2, target;
    DevBuf<int> done, iters, brk;
    DevBuf<float2> U32;
    DevBuf<unsigned char> scratch;
    for (DevBuf<VT> *b : {&r, &p, &Dp, &Dr, &Mp, &sres, &d}) WFQ_TRY(b->alloc(ctx, nc, s));
    for (DevBuf<double2> *b : {&rho, &sigma, &alpha, &beta, &cd, &ca}) WFQ_TRY(b->alloc(ctx, cc, s));
    for (DevBuf<double> *b : {&tau, &theta, &c2, &target}) WFQ_TRY(b->alloc(ctx, cc, s));
    for (DevBuf<int> *b : {&done, &iters, &brk}) WFQ_TRY(b->alloc(ctx, cc, s));
    if (mixed) WFQ_TRY(scratch.alloc(ctx, mixed_scratch_bytes(g, cc), s));
    WFQ_CUDA(cudaMemsetAsync(iters.ptr, 0, sizeof(int) * cc, s));
    WFQ_CUDA(cudaMemsetAsync(brk.ptr, 0, sizeof(int) * cc, s));
    WFQ_CUDA(cudaMemsetAsync(a.q, 0, sizeof(double2) * nc, s));
    QmrDev q{cc, rho.ptr, sigma.ptr, alpha.ptr, beta.ptr, tau.ptr, theta.ptr, c2.ptr,
             cd.ptr, ca.ptr, target.ptr, done.ptr, iters.ptr, brk.ptr};
    const ColGrid cg = cm.cg;
    const double inner_red = mixed ? 1e-6 : 0.0;

    // U = D v in the working precision
    auto dmul = [&](const VT *v, VT *u) -> int {
        if (mixed)
            return d_apply_mixed(g, cc, reinterpret_cast<const float2 *>(v), reinterpret_cast<float2 *>(u),
                                 scratch.ptr, s);
        return d_apply_fp64(g, cc, reinterpret_cast<const double2 *>(v), reinterpret_cast<double2 *>(u), s);
    };
    auto sparse = [&](const VT *u, const VT *x, VT *y) -> int {
        if (mixed)
            return sparse_shift_fp32(g, cc, reinterpret_cast<const float2 *>(u), reinterpret_cast<const float2 *>(x),
                                     cm.z.ptr, reinterpret_cast<float2 *>(y), s);
        return sparse_shift_fp64(g, cc, reinterpret_cast<const double2 *>(u), reinterpret_cast<const double2 *>(x),
                                 cm.z.ptr, reinterpret_cast<double2 *>(y), s);
    };

    std::vector<int> done_h(cc), conv_h(cc), brk_h(cc);
    int total = 0, cycles = 0;
    bool breakdown_any = false;
    for (;;) {
        if (cycles == 0) {
            WFQ_CUDA(cudaMemcpyAsync(cm.r.ptr, cm.B.ptr, sizeof(double2) * nc, cudaMemcpyDeviceToDevice, s));
            WFQ_CUDA(cudaMemcpyAsync(cm.rnorm.ptr, cm.bnorm.ptr, sizeof(double2) * cc, cudaMemcpyDeviceToDevice, s));
        } else {
            WFQ_TRY(cm.true_residual(a.q));
        }
        k_qmr_restart_cols<<<nblocks(cc), 256, 0, s>>>(cc, cm.rnorm.ptr, cm.bnorm.ptr, a.rel_tol, inner_red, q,
                                                       cm.converged.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        WFQ_CUDA(cudaMemcpyAsync(conv_h.data(), cm.converged.ptr, sizeof(int) * cc, cudaMemcpyDeviceToHost, s));
        WFQ_CUDA(cudaMemcpyAsync(brk_h.data(), brk.ptr, sizeof(int) * cc, cudaMemcpyDeviceToHost, s));
        WFQ_TRY(check_device_error(g->ctx, s));
        bool unfinished = false;
        for (int64_t c = 0; c < cc; ++c)
            if (!conv_h[c] && !brk_h[c]) unfinished = true;
        if (!unfinished || total >= a.max_iter) break;
        // columns that broke down stay out of later restarts
        k_qmr_restart_vec<VT><<<nblocks(nc), 256, 0, s>>>(nc, cc, cm.r.ptr, cm.converged.ptr, r.ptr, p.ptr,
                                                          sres.ptr, d.ptr); note_launch();
        WFQ_CUDA(cudaGetLastError());
        WFQ_TRY(dmul(r.ptr, Dr.ptr));
        WFQ_CUDA(cudaMemcpyAsync(Dp.ptr, Dr.ptr, sizeof(VT) * nc, cudaMemcpyDeviceToDevice, s));
        k_qmr_red<VT><<<cg.nblk, 256, 0, s>>>(n, cc, cg.cx, cg.ry, QF_RESTART, r.ptr, Dr.ptr, cm.red, q); note_launch();
        WFQ_CUDA(cudaGetLastError());
        int since = 0;
        for (;;) {
            if (total >= a.max_iter) break;
            WFQ_TRY(sparse(Dp.ptr, p.ptr, Mp.ptr));  // M p = (Kbar - P) D p - z p
            k_qmr_red<VT><<<cg.nblk, 256, 0, s>>>(n, cc, cg.cx, cg.ry, QF_SIGMA, Dp.ptr, Mp.ptr, cm.red, q); note_launch();
            k_qmr_r<VT><<<nblocks(nc), 256, 0, s>>>(nc, cc, r.ptr, Mp.ptr, q); note_launch();
            k_qmr_red<VT><<<cg.nblk, 256, 0, s>>>(n, cc, cg.cx, cg.ry, QF_RNORM, r.ptr, nullptr, cm.red, q); note_launch();
            k_qmr_dxs<VT><<<nblocks(nc), 256, 0, s>>>(nc, cc, d.ptr, p.ptr, a.q, sres.ptr, r.ptr, q); note_launch();
            k_qmr_red<VT><<<cg.nblk, 256, 0, s>>>(n, cc, cg.cx, cg.ry, QF_SNORM, sres.ptr, nullptr, cm.red, q); note_launch();
            WFQ_CUDA(cudaGetLastError());
            ++total;
            ++since;
            WFQ_CUDA(cudaMemcpyAsync(done_h.data(), done.ptr, sizeof(int) * cc, cudaMemcpyDeviceToHost, s));
            WFQ_CUDA(cudaStreamSynchronize(s));
            bool all_done = std::all_of(done_h.begin(), done_h.end(), [](int v) { return v != 0; });
            if (all_done) break;
            if (mixed && a.refine_every > 0 && since >= a.refine_every) break;
            WFQ_TRY(dmul(r.ptr, Dr.ptr));                 // the one D product of the iteration
            k_qmr_red<VT><<<cg.nblk, 256, 0, s>>>(n, cc, cg.cx, cg.ry, QF_RHO, r.ptr, Dr.ptr, cm.red, q); note_launch();
            k_qmr_p<VT><<<nblocks(nc), 256, 0, s>>>(nc, cc, p.ptr, Dp.ptr, r.ptr, Dr.ptr, q); note_launch();
            WFQ_CUDA(cudaGetLastError());
        }
        ++cycles;
    }
    WFQ_CUDA(cudaMemcpyAsync(brk_h.data(), brk.ptr, sizeof(int) * cc, cudaMemcpyDeviceToHost, s));
    if (cycles > 0) WFQ_TRY(cm.true_residual(a.q));
    std::vector<int> it(cc);
    WFQ_CUDA(cudaMemcpyAsync(it.data(), iters.ptr, sizeof(int) * cc, cudaMemcpyDeviceToHost, s));
    WFQ_CUDA(cudaStreamSynchronize(s));
    for (int64_t c = 0; c < cc; ++c) breakdown_any = breakdown_any || brk_h[c];
    return fill_stats(a, cm, it, cycles, 0, breakdown_any, brk_h);
}

int solve_qmr(wfq_geom *g, const SolveArgs &a, cudaStream_t s) {
    if (a.prec == WFQ_PREC_MIXED) return qmr_impl<float2>(g, a, s);
    return qmr_impl<double2>(g, a, s);
}

}  // namespace wfq
