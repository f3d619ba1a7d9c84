// Structure-dependent set-up: Kbar neighbour list (Eq. 6, Eq. 9), P (Eq. 16),
// D (Eq. 3 with the widths of Eq. 4), right-hand sides (Eq. 2, Eq. 13) and the
// polarizability reduction (Eq. 28).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.h"

namespace wfq {

// ------------------------------------------------------------------ Kbar CSR (host)

// Distance beyond which 1 - f(r) < eps (Eq. 6): 1/(1 + exp(d (r/(s r0) - 1))) >= eps
// <=> r <= s r0 (1 + ln(1/eps - 1) / d).
static double kbar_cutoff_radius(const wfq_params &p) {
    if (p.cutoff_eps <= 0.0) return INFINITY;
    return p.s_fermi * p.r0 * (1.0 + std::log(1.0 / p.cutoff_eps - 1.0) / p.d_fermi);
}

static inline double one_minus_fermi(const wfq_params &p, double r) {
    return 1.0 / (1.0 + std::exp(p.d_fermi * (r / (p.s_fermi * p.r0) - 1.0)));
}

int build_kbar_csr(int64_t n, const double *xyz, const wfq_params &p,
                   std::vector<int64_t> &rowptr, std::vector<int32_t> &col,
                   std::vector<double> &val) {
    const double rc = kbar_cutoff_radius(p);
    const double min_sep = 1e-8;
    rowptr.assign(n + 1, 0);
    std::vector<std::vector<std::pair<int32_t, double>>> rows(n);

    // Returns false if a coincident pair is found.
    auto scan_pair = [&](int64_t i, int64_t j, std::vector<std::pair<int32_t, double>> &out) {
        double dx = xyz[3 * i] - xyz[3 * j], dy = xyz[3 * i + 1] - xyz[3 * j + 1],
               dz = xyz[3 * i + 2] - xyz[3 * j + 2];
        double r = std::sqrt(dx * dx + dy * dy + dz * dz);
        if (r < min_sep) return false;
        if (r > rc) return true;
        double omf = one_minus_fermi(p, r);
        if (omf >= p.cutoff_eps) out.emplace_back(static_cast<int32_t>(j), omf * p.area / r);
        return true;
    };

    bool dup = false;
    if (!std::isfinite(rc)) {
        // every pair is a neighbour: dense Kbar (small systems only)
#pragma omp parallel for schedule(dynamic, 32) reduction(|| : dup)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j)
                if (j != i && !scan_pair(i, j, rows[i])) dup = true;
    } else {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], xyz[3 * i + k]);
                hi[k] = std::max(hi[k], xyz[3 * i + k]);
            }
        double cell = rc;
        int64_t dims[3];
        for (;;) {
            for (int k = 0; k < 3; ++k)
                dims[k] = std::max<int64_t>(1, (int64_t)std::floor((hi[k] - lo[k]) / cell) + 1);
            if (dims[0] * dims[1] * dims[2] <= (int64_t)1 << 26) break;
            cell *= 2.0;
        }
        const int64_t ncell = dims[0] * dims[1] * dims[2];
        auto cell_of = [&](int64_t i, int64_t c[3]) {
            for (int k = 0; k < 3; ++k)
                c[k] = std::min<int64_t>(dims[k] - 1, (int64_t)((xyz[3 * i + k] - lo[k]) / cell));
        };
        std::vector<int64_t> start(ncell + 1, 0), order(n);
        for (int64_t i = 0; i < n; ++i) {
            int64_t c[3];
            cell_of(i, c);
            start[(c[2] * dims[1] + c[1]) * dims[0] + c[0] + 1]++;
        }
        for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < n; ++i) {
            int64_t c[3];
            cell_of(i, c);
            order[fill[(c[2] * dims[1] + c[1]) * dims[0] + c[0]]++] = i;
        }
#pragma omp parallel for schedule(dynamic, 64) reduction(|| : dup)
        for (int64_t i = 0; i < n; ++i) {
            int64_t c[3];
            cell_of(i, c);
            for (int64_t z = std::max<int64_t>(0, c[2] - 1); z <= std::min(dims[2] - 1, c[2] + 1); ++z)
                for (int64_t y = std::max<int64_t>(0, c[1] - 1); y <= std::min(dims[1] - 1, c[1] + 1); ++y)
                    for (int64_t x = std::max<int64_t>(0, c[0] - 1); x <= std::min(dims[0] - 1, c[0] + 1); ++x) {
                        int64_t cid = (z * dims[1] + y) * dims[0] + x;
                        for (int64_t t = start[cid]; t < start[cid + 1]; ++t) {
                            int64_t j = order[t];
                            if (j != i && !scan_pair(i, j, rows[i])) dup = true;
                        }
                    }
            std::sort(rows[i].begin(), rows[i].end());
        }
    }
    if (dup) return fail(WFQ_EINVAL, "two atoms closer than 1e-8 bohr (r_ij = 0 makes Eq. 3 undefined)");
    for (int64_t i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + (int64_t)rows[i].size();
    col.resize(rowptr[n]);
    val.resize(rowptr[n]);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t q = rowptr[i];
        for (auto &e : rows[i]) {
            col[q] = e.first;
            val[q] = e.second;
            ++q;
        }
    }
    return WFQ_OK;
}

// ------------------------------------------------------------------ D build (device)

// Entry (i, j) of Eq. 3.  For r >= 6 sigma, erfc(r/sigma) < 2^-54 and erf rounds to
// exactly 1 in FP64, so 1/r is returned without evaluating erf (same value).
__device__ __forceinline__ double d_entry64(atom64_t a, atom64_t b, double eta_i, bool diag) {
    if (diag) return eta_i;
    double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    double r2 = dx * dx + dy * dy + dz * dz;
    double r = sqrt(r2);
    double s2 = a.w * a.w + b.w * b.w;
    if (r2 >= 36.0 * s2) return 1.0 / r;
    return erf(r / sqrt(s2)) / r;
}

// One thread per (i, j) with j fastest; writes the FP64 D, the bf16 hi/lo planes
// (hi = bf16(D), lo = bf16(D - hi), zero outside n x n) and / or the FP32 hi/lo planes
// (fh = fl32(D), fl = fl32(D - fh), rows of ldf >= n entries, zero for j >= n).
__global__ void k_build_d(const atom64_t *__restrict__ atom, const double *__restrict__ eta,
                          int64_t n, int64_t npad, int64_t lim, double *__restrict__ D64,
                          __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
                          int64_t ldf, float *__restrict__ fh, float *__restrict__ fl) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= lim || j >= lim) return;
    double v = 0.0;
    if (i < n && j < n) v = d_entry64(atom[i], atom[j], eta[i], i == j);
    if (D64 && i < n && j < n) D64[i * n + j] = v;
    if (fh && i < n && j < ldf) {
        const float h = (float)v;
        fh[i * ldf + j] = h;
        fl[i * ldf + j] = (float)(v - (double)h);
    }
    if (hi) {
        __nv_bfloat16 h = __double2bfloat16(v);
        __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
        hi[i * npad + j] = h;
        lo[i * npad + j] = l;
    }
}

// BEM operator (Eq. 22 in charge form), one thread per (i, j) with j fastest, into the same
// storages as D (FP64, bf16 hi/lo planes zero-padded to npad, FP32 hi/lo planes of ldf
// columns): A_ij = a_i n_i . (r_i - r_j) / |r_i - r_j|^3, A_ii = the element's self
// coefficient.  *close is set when two distinct elements lie closer than 1e-8 bohr.
__global__ void k_build_bem(const elem64_t *__restrict__ el, int64_t n, int64_t npad, int64_t lim,
                            double *__restrict__ D64, __nv_bfloat16 *__restrict__ hi,
                            __nv_bfloat16 *__restrict__ lo, int64_t ldf, float *__restrict__ fh,
                            float *__restrict__ fl, int *__restrict__ close) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= lim || j >= lim) return;
    double v = 0.0;
    if (i < n && j < n) {
        const elem64_t a = el[i];
        if (i == j) {
            v = a.self;
        } else {
            const elem64_t b = el[j];
            const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < 1e-16) {
                atomicOr(close, 1);
            } else {
                v = a.area * (a.nx * dx + a.ny * dy + a.nz * dz) / (r2 * sqrt(r2));
            }
        }
    }
    if (D64 && i < n && j < n) D64[i * n + j] = v;
    if (fh && i < n && j < ldf) {
        const float h = (float)v;
        fh[i * ldf + j] = h;
        fl[i * ldf + j] = (float)(v - (double)h);
    }
    if (hi) {
        __nv_bfloat16 h = __double2bfloat16(v);
        __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
        hi[i * npad + j] = h;
        lo[i * npad + j] = l;
    }
}

int launch_build_bem(const wfq_geom *g, int *close, cudaStream_t s) {
    const int64_t lim = g->Dhi ? g->npad : (g->Dfh ? g->ldf : g->n);   // ldf <= npad
    dim3 block(64, 4);
    dim3 grid((unsigned)((lim + 63) / 64), (unsigned)((lim + 3) / 4));
    if (grid.y > 65535u) return fail(WFQ_EUNSUPPORTED, "stored BEM operator with more than 262140 rows");
    k_build_bem<<<grid, block, 0, s>>>(g->elem, g->n, g->npad, lim, g->D64, g->Dhi, g->Dlo, g->ldf, g->Dfh, g->Dfl,
                                       close); note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

// Upper-triangle tiles of the FP32 pair D: block (x, y) fills 256 entries of tile row
// I = y; entry q of the row's run of tiles is tile J = I + q / 4096, element q % 4096.
__global__ void k_build_dsym(const atom64_t *__restrict__ atom, const double *__restrict__ eta, int64_t n,
                             int64_t T, float *__restrict__ Dsym) {
    const int64_t I = blockIdx.y;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t J = I + q / (kSymTile * kSymTile);
    if (J >= T) return;
    const int64_t e = q % (kSymTile * kSymTile);
    const int64_t i = I * kSymTile + e / kSymTile, j = J * kSymTile + e % kSymTile;
    const double v = (i < n && j < n) ? d_entry64(atom[i], atom[j], eta[i], i == j) : 0.0;
    float *tile = Dsym + sym_tile(I, J, T) * 2 * kSymTile * kSymTile;
    const float h = (float)v;
    tile[e] = h;
    tile[kSymTile * kSymTile + e] = (float)(v - (double)h);
}

int launch_build_d(const wfq_geom *g, cudaStream_t s) {
    if (g->Dsym) {
        const int64_t T = g->sym_nt;
        if (T > 65535) return fail(WFQ_EUNSUPPORTED, "symmetric tiled D with more than 65535 tile rows");
        dim3 grid((unsigned)((T * kSymTile * kSymTile + 255) / 256), (unsigned)T);
        k_build_dsym<<<grid, 256, 0, s>>>(g->atom64, g->eta, g->n, T, g->Dsym); note_launch();
        WFQ_CUDA(cudaGetLastError());
    }
    if (!g->D64 && !g->Dhi && !g->Dfh) return WFQ_OK;
    const int64_t lim = g->Dhi ? g->npad : (g->Dfh ? g->ldf : g->n);   // ldf <= npad
    dim3 block(64, 4);
    dim3 grid((unsigned)((lim + 63) / 64), (unsigned)((lim + 3) / 4));
    if (grid.y > 65535u) return fail(WFQ_EUNSUPPORTED, "stored D with more than 262140 rows");
    k_build_d<<<grid, block, 0, s>>>(g->atom64, g->eta, g->n, g->npad, lim, g->D64, g->Dhi, g->Dlo, g->ldf, g->Dfh,
                                     g->Dfl); note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

// ------------------------------------------------------------------ RHS (Eq. 13)

// R[i][d] = sum_j (V_i - V_j) Kbar_ij with V = -E0 (r . dir_d).
__global__ void k_rhs(int64_t n, const double *__restrict__ xyz, const int64_t *__restrict__ rowptr,
                      const int32_t *__restrict__ col, const double *__restrict__ val, int ndir,
                      const double *__restrict__ dirs, double E0, double *__restrict__ R) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int d = 0; d < ndir; ++d) {
        double kx = dirs[3 * d], ky = dirs[3 * d + 1], kz = dirs[3 * d + 2];
        double Vi = -E0 * (xyz[3 * i] * kx + xyz[3 * i + 1] * ky + xyz[3 * i + 2] * kz);
        double acc = 0.0;
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            int64_t j = col[q];
            double Vj = -E0 * (xyz[3 * j] * kx + xyz[3 * j + 1] * ky + xyz[3 * j + 2] * kz);
            acc += (Vi - Vj) * val[q];
        }
        R[i * ndir + d] = acc;
    }
}

// BEM: R[i][d] = -E0 a_i (n_i . dir_d), element i's area times the normal derivative of
// phi = -E0 dir_d . r (Eq. 21 with the sign that makes q the physical charge).
__global__ void k_rhs_bem(int64_t n, const elem64_t *__restrict__ el, int ndir, const double *__restrict__ dirs,
                          double E0, double *__restrict__ R) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const elem64_t e = el[i];
    for (int d = 0; d < ndir; ++d)
        R[i * ndir + d] = -E0 * e.area * (e.nx * dirs[3 * d] + e.ny * dirs[3 * d + 1] + e.nz * dirs[3 * d + 2]);
}

int launch_rhs(const wfq_geom *g, int ndir, const double *dirs_dev, double E0, double *R,
               cudaStream_t s) {
    int64_t n = g->n;
    if (g->op == OP_BEM) {
        k_rhs_bem<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, g->elem, ndir, dirs_dev, E0, R); note_launch();
        WFQ_CUDA(cudaGetLastError());
        return WFQ_OK;
    }
    k_rhs<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, g->xyz, g->rowptr, g->col, g->val64, ndir,
                                                     dirs_dev, E0, R); note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

// ------------------------------------------------------------------ alpha (Eq. 28)

// Pass 1: per-block partial sums of q_i r_{i,k} for every column (fixed order).
__global__ void k_alpha_partial(int64_t n, int64_t ncols, const double2 *__restrict__ q,
                                const double *__restrict__ xyz, double2 *__restrict__ part) {
    // blockIdx.y: column chunk of blockDim.x columns; blockIdx.x: atom chunk
    int64_t c = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    if (c >= ncols) return;
    double2 a[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t i = i0; i < i1; ++i) {
        double2 v = q[i * ncols + c];
        for (int k = 0; k < 3; ++k) {
            double x = xyz[3 * i + k];
            a[k].x += v.x * x;
            a[k].y += v.y * x;
        }
    }
    for (int k = 0; k < 3; ++k) part[((int64_t)blockIdx.x * ncols + c) * 3 + k] = a[k];
}

__global__ void k_alpha_final(int nblk, int64_t ncols, const double2 *__restrict__ part, double E0,
                              double2 *__restrict__ alpha) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncols * 3) return;
    double2 s = {0, 0};
    for (int b = 0; b < nblk; ++b) {
        double2 v = part[(int64_t)b * ncols * 3 + t];
        s.x += v.x;
        s.y += v.y;
    }
    alpha[t] = make_double2(s.x / E0, s.y / E0);
}

int launch_polarizability(const wfq_geom *g, int64_t ncols, const double2 *q, double E0,
                          double2 *alpha_dev, cudaStream_t s) {
    const int nblk = 256;
    DevBuf<double2> part;
    WFQ_TRY(part.alloc(g->ctx, (size_t)nblk * ncols * 3, s));
    dim3 grid(nblk, (unsigned)((ncols + 63) / 64));
    k_alpha_partial<<<grid, 64, 0, s>>>(g->n, ncols, q, g->xyz, part.ptr); note_launch();
    WFQ_CUDA(cudaGetLastError());
    k_alpha_final<<<(unsigned)((ncols * 3 + 127) / 128), 128, 0, s>>>(nblk, ncols, part.ptr, E0,
                                                                       alpha_dev); note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

// Eq. 28 and Eq. 29 from the polarizability of each column: with the field along
// k = dir / |dir| at amplitude E0 |dir|, sum_i (r_i . k) Im q_i / (E0 |dir|) = Im(dir . alpha_c) / |dir|^2
// (alpha_c = sum_i q_i r_i / E0), so sigma_{f,d} = (4 pi w_f / c) Im(dir_d . alpha_c) / |dir_d|^2.
// One thread per frequency: its ndir columns and their mean (Eq. 29 for an orthonormal triad).
__global__ void k_cross_section(int64_t nfreq, int ndir, const double *__restrict__ omega,
                                const double *__restrict__ dirs, const double2 *__restrict__ alpha,
                                double *__restrict__ sigma, double *__restrict__ sigma_iso) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfreq) return;
    const double c_au = 137.035999084;   // speed of light in atomic units (CODATA 2018)
    const double pref = 4.0 * 3.14159265358979323846 * omega[f] / c_au;
    double mean = 0.0;
    for (int d = 0; d < ndir; ++d) {
        const double *k = dirs + 3 * d;
        const double2 *a = alpha + (f * ndir + d) * 3;
        const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        const double im = k[0] * a[0].y + k[1] * a[1].y + k[2] * a[2].y;
        const double s = pref * im / kk;
        sigma[f * ndir + d] = s;
        mean += s;
    }
    if (sigma_iso) sigma_iso[f] = mean / ndir;
}

int launch_cross_section(const wfq_geom *g, int64_t nfreq, int ndir, const double *omega_dev,
                         const double *dirs_dev, const double2 *q, double E0, double *sigma_dev,
                         double *sigma_iso_dev, cudaStream_t s) {
    const int64_t ncols = nfreq * ndir;
    DevBuf<double2> alpha;
    WFQ_TRY(alpha.alloc(g->ctx, (size_t)ncols * 3, s));
    WFQ_TRY(launch_polarizability(g, ncols, q, E0, alpha.ptr, s));
    k_cross_section<<<(unsigned)((nfreq + 127) / 128), 128, 0, s>>>(nfreq, ndir, omega_dev, dirs_dev, alpha.ptr,
                                                                     sigma_dev, sigma_iso_dev);
    note_launch();
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

}  // namespace wfq
