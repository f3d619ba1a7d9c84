// Internal declarations of libwfq (not part of the C ABI; see include/wfq.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/wfq.h"

namespace wfq {

// ------------------------------------------------------------------ errors

void set_error(const std::string &msg);
// Solver progress on stderr (one line per restart cycle, escalation and continuation) when
// the environment variable WFQ_TRACE is set and not "0"; off otherwise.
bool trace_on();
void trace(const char *fmt, ...) __attribute__((format(printf, 1, 2)));
const char *get_error();

struct Status {
    int code = WFQ_OK;
    explicit operator bool() const { return code != WFQ_OK; }
};

#define WFQ_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ::wfq::set_error(std::string(#call) + ": " + cudaGetErrorString(e_) + " at " + \
                             __FILE__ + ":" + std::to_string(__LINE__));                   \
            return WFQ_ECUDA;                                                              \
        }                                                                                  \
    } while (0)

#define WFQ_TRY(expr)                 \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != WFQ_OK) return rc_; \
    } while (0)

inline int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------------ handles

// Tensor-core tile geometry of the stored bf16 D planes: rows and columns padded
// to a multiple of kTilePad with zero entries.
constexpr int64_t kTilePad = 128;

// Symmetric tiled D (WFQ_STORE_F32X2_SYM): edge of a tile, and the work item of one CTA of
// the symmetric product -- tiles J0 .. J1 - 1 of tile row I.
constexpr int64_t kSymTile = 64;
struct SymItem {
    int I, J0, J1, pad;
};
// index of tile (I, J), I <= J, in the row-ordered upper triangle of T x T tiles
__host__ __device__ inline int64_t sym_tile(int64_t I, int64_t J, int64_t T) { return I * T - I * (I - 1) / 2 + (J - I); }

// Per-atom record for the FP64 kernels: position and Gaussian width (Eq. 4).
struct __align__(32) atom64_t {
    double x, y, z, w;
};

// Operator family of a geometry: the omega-FQ operator A = (Kbar - P) D (Eq. 14, 17), or
// the continuum BEM operator of Eq. 21-22 in charge form (A = F scaled by the element
// areas, no sparse term, z = -Lambda(w)).
enum OpKind { OP_WFQ = 0, OP_BEM = 1 };

// Per-element record of the BEM operator: collocation point, outward unit normal, area and
// self coefficient (the principal value of Eq. 22 over the element itself).
struct __align__(64) elem64_t {
    double x, y, z, nx, ny, nz, area, self;
};

// The frequency-dependent shift z(w) of a geometry's operator family.
struct ShiftModel {
    int op;
    double n0, tau;                       // omega-FQ, Eq. 12
    double eps_out, eps_inf, wp, gamma;   // BEM: Drude particle in a uniform host
};

// omega-FQ: z = -(w / (2 n0 tau)) (w tau + i)  (Eq. 12).
// BEM: z = -Lambda(w) = -2 pi (eps_out + eps_in) / (eps_out - eps_in)  (Eq. 21), with
// eps_in = eps_inf - wp^2 / (w (w + i gamma)) = eps_inf - wp^2 / (w^2 + gamma^2)
//          + i wp^2 gamma / (w (w^2 + gamma^2)).
__host__ __device__ inline double2 z_eval(const ShiftModel &m, double w) {
    if (m.op == OP_BEM) {
        const double den = w * w + m.gamma * m.gamma;
        const double er = m.eps_inf - m.wp * m.wp / den;
        const double ei = m.wp * m.wp * m.gamma / (w * den);
        const double ar = m.eps_out + er, ai = ei;     // eps_out + eps_in
        const double br = m.eps_out - er, bi = -ei;    // eps_out - eps_in
        const double bb = br * br + bi * bi;
        const double two_pi = 6.283185307179586476925286766559;
        return make_double2(-two_pi * (ar * br + ai * bi) / bb, -two_pi * (ai * br - ar * bi) / bb);
    }
    const double f = -w / (2.0 * m.n0 * m.tau);
    return make_double2(f * w * m.tau, f);
}

}  // namespace wfq

namespace wfq {

// Event-pair timing of selected kernel classes (wfq_profile / wfq_profile_read).
struct KernelTimer {
    std::mutex mu;
    bool enabled = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[WFQ_KT_COUNT];
    std::vector<cudaEvent_t> pool;
    std::vector<double> pending_work[WFQ_KT_COUNT];
    int64_t launches[WFQ_KT_COUNT] = {};
    double ms[WFQ_KT_COUNT] = {};
    double work[WFQ_KT_COUNT] = {};
    cudaEvent_t get();
    void collect();
    void reset();
    ~KernelTimer();
};

}  // namespace wfq

struct wfq_ctx {
    int device = 0;
    int num_sms = 0;
    cudaMemPool_t pool = nullptr;
    int *dev_err = nullptr;   // device flag: non-zero after a bounded wait in a kernel gave up
    wfq::KernelTimer timer;
    // autotuner results: kernel tiling chosen by timing, per problem key (kept across
    // geometries of the same shape)
    std::mutex tune_mu;
    std::map<int64_t, int> tuned;
};

namespace wfq {
struct Fmm;   // fast-multipole tree and operators (fmm.cu)
}

struct wfq_geom {
    wfq_ctx *ctx = nullptr;
    int op = wfq::OP_WFQ;   // operator family (wfq::OpKind)
    int64_t n = 0;      // atoms (BEM: surface elements)
    int64_t npad = 0;   // n rounded up to kTilePad (bf16 plane dimension)
    wfq_params p{};
    wfq_bem_params bem{};   // BEM geometries only
    uint32_t store = 0;
    int64_t nnz = 0;
    size_t bytes = 0;   // device bytes held

    // per-atom (device)
    double *xyz = nullptr;      // n x 3
    wfq::atom64_t *atom64 = nullptr;  // (x, y, z, width), n
    float4 *atom32 = nullptr;   // (x, y, z, width), npad (padding: far away, width 1)
    float4 *atom32p = nullptr;  // the same records by atom pairs (2k, 2k + 1): (x0, x1, y0, y1),
                                // (z0, z1, w0, w1) -- one float4 per atom, npad; the matrix-free
                                // generator reads them as packed FP32x2 operands
    float4 *atomdf = nullptr;   // 2 per atom: (xh, xl, yh, yl), (zh, zl, width, 0) float pairs
    double *eta = nullptr;      // n
    wfq::elem64_t *elem = nullptr;   // BEM geometries: n element records

    // Kbar CSR (device)
    int64_t *rowptr = nullptr;  // n + 1
    int32_t *col = nullptr;     // nnz
    double *val64 = nullptr;    // nnz
    float *val32 = nullptr;     // nnz

    // D storages (device)
    double *D64 = nullptr;      // n x n row-major (ld = n)
    __nv_bfloat16 *Dhi = nullptr;  // npad x npad row-major
    __nv_bfloat16 *Dlo = nullptr;
    float *Dfh = nullptr;       // n x ldf row-major: fl32(D_ij) (zero for j >= n)
    float *Dfl = nullptr;       // n x ldf row-major: fl32(D_ij - Dfh_ij)
    int64_t ldf = 0;            // n rounded up to 128 (512-byte rows; the GEMV steps 128 columns)
    // upper-triangle 64 x 64 tiles of the FP32 pairs (WFQ_STORE_F32X2_SYM)
    float *Dsym = nullptr;      // tile t(I, J): 4096 hi then 4096 lo floats, row-major
    int64_t sym_nt = 0;         // tiles per side, ceil(n / 64)
    wfq::SymItem *sym_items = nullptr;   // work items of the symmetric product (device)
    int64_t sym_nitems = 0;
    int *sym_item_start = nullptr;       // [sym_nt + 1]: first item of each tile row (device)
    wfq::Fmm *fmm = nullptr;             // wfq_fmm_build: tree and operators of the FMM product
};

namespace wfq {

// ------------------------------------------------------------------ memory

// Stream-ordered allocation from the context's pool.
int dalloc(wfq_ctx *ctx, void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);

template <class T>
struct DevBuf {
    T *ptr = nullptr;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() {
        if (ptr) dfree(ptr, s);
    }
    int alloc(wfq_ctx *ctx, size_t count, cudaStream_t stream) {
        s = stream;
        return dalloc(ctx, reinterpret_cast<void **>(&ptr), count * sizeof(T), stream);
    }
};

// Counts kernel launches made by the library (wfq_kernel_launches).
void note_launch();

// Records start/end events around the launches made in its scope when timing is on.
struct KScope {
    wfq_ctx *ctx;
    int kind;
    cudaStream_t s;
    double work;
    cudaEvent_t e0 = nullptr;
    KScope(wfq_ctx *c, int k, cudaStream_t st, double w = 0.0);
    ~KScope();
};

// WFQ_ETIMEOUT (and clears the flag) if a kernel reported a bounded wait that gave up.
int check_device_error(wfq_ctx *ctx, cudaStream_t s);

// True if p is a device (or managed) pointer usable by kernels.
// 1: device memory of `device` (or managed memory); 0: host memory; -1: device memory of
// another device (kernels of this context must not touch it).
int device_ptr_on(const void *p, int device);

// ------------------------------------------------------------------ geometry build

int build_kbar_csr(int64_t n, const double *xyz, const wfq_params &p, std::vector<int64_t> &rowptr,
                   std::vector<int32_t> &col, std::vector<double> &val);

int launch_build_d(const wfq_geom *g, cudaStream_t s);
// BEM geometries: the operator's entries into the requested storages; *close is set
// non-zero (device int) when two elements lie closer than 1e-8 bohr.
int launch_build_bem(const wfq_geom *g, int *close, cudaStream_t s);
int launch_rhs(const wfq_geom *g, int ndir, const double *dirs_dev, double E0, double *R,
               cudaStream_t s);
// sigma_{f,d} (Eq. 28) of the nfreq x ndir columns of q, and their per-frequency mean (Eq. 29)
// when sigma_iso_dev is not null.  omega_dev, dirs_dev: device copies of the caller's arrays.
int launch_cross_section(const wfq_geom *g, int64_t nfreq, int ndir, const double *omega_dev,
                         const double *dirs_dev, const double2 *q, double E0, double *sigma_dev,
                         double *sigma_iso_dev, cudaStream_t s);
int launch_polarizability(const wfq_geom *g, int64_t ncols, const double2 *q, double E0,
                          double2 *alpha_dev, cudaStream_t s);

// ------------------------------------------------------------------ operator pieces
// Block vectors are atom-major: element (atom i, complex column c) at i * cc + c.

// U = D X in FP64 (stored FP64 D if present, else recomputed from the coordinates).
int d_apply_fp64(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s);

// U = D X with double-float products (FP64 operands split into float pairs, about 48
// significant bits) when the FP64 D is stored and there are more than 4 columns; else
// the FP64 kernels.  Used for the refinement residual of mixed-precision solves.
int d_apply_df(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s);

// U = D X for at most 4 complex columns with double-float products (~2^-48 per product)
// from the stored float pairs (full planes or symmetric tiles) -- the FP64-grade product of
// geometries that store no FP64 D (shifted.cu).
int d_apply_pairs_df(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s);
// The same for a geometry with no stored D: D regenerated per product in double-float
// (the shifted solver's matrix-free GEMV), at most 4 complex columns.
int d_apply_mf_gemv_df(const wfq_geom *g, int64_t cc, const double2 *X, double2 *U, cudaStream_t s);

// U = D X with 3 bf16 products and FP32 accumulation: stored bf16 planes when present,
// else tiles generated from the coordinates (matrix-free).
// scratch: at least mixed_scratch_bytes(g, cc) bytes of device memory.
size_t mixed_scratch_bytes(const wfq_geom *g, int64_t cc);
int d_apply_mixed(const wfq_geom *g, int64_t cc, const float2 *X, float2 *U, void *scratch,
                  cudaStream_t s);

// Fast-multipole D product (fmm.cu): build the tree and operators of an order, free them,
// their device bytes, the tree summary of wfq_fmm_info, and U = D X with it (FP32).
int fmm_build(wfq_geom *g, int order, Fmm **out);
void fmm_free(Fmm *f);
size_t fmm_bytes(const Fmm *f);
void fmm_info(const Fmm *f, int64_t *out);
int d_apply_fmm(const wfq_geom *g, int64_t cc, const float2 *X, float2 *U, cudaStream_t s);

// Y = Kbar U - P U - z_c X   (z: device, cc values); BEM geometries: Y = U - z_c X
int sparse_shift_fp64(const wfq_geom *g, int64_t cc, const double2 *U, const double2 *X,
                      const double2 *z, double2 *Y, cudaStream_t s);
int sparse_shift_fp32(const wfq_geom *g, int64_t cc, const float2 *U, const float2 *X,
                      const double2 *z, float2 *Y, cudaStream_t s);

// U[n x ldu] (fp32, row-major) = Dhi.Xhi + Dhi.Xlo + Dlo.Xhi where Xhi/Xlo are
// [cpad x npad] bf16 (K-major), cpad a multiple of 64 and >= ldu.  Only rows < n and
// columns < ldu of U are written.
int gemm_3xbf16(const wfq_geom *g, int64_t cpad, const __nv_bfloat16 *Xhi,
                const __nv_bfloat16 *Xlo, float *U, int64_t ldu, cudaStream_t s);

// As gemm_3xbf16 with the D tiles generated from the atom records (matrix-free).
int gemm_3xbf16_mf(const wfq_geom *g, int64_t cpad, const __nv_bfloat16 *Xhi,
                   const __nv_bfloat16 *Xlo, float *U, int64_t ldu, cudaStream_t s);

// ------------------------------------------------------------------ solvers

struct SolveArgs {
    int64_t nfreq = 0;
    const double *omega = nullptr;  // host
    int ndir = 0;
    const double *dirs = nullptr;   // host, ndir x 3
    // Optional explicit column list (used by the server when it merges requests): column
    // c solves at frequency col_omega[c] with field direction dirs[col_dir[c]]; ncols columns.
    // When null, the columns are the product nfreq x ndir (c = f * ndir + d).
    const double *col_omega = nullptr;
    const int *col_dir = nullptr;
    int64_t ncols = 0;
    double E0 = 1.0;
    int m = 0;
    double rel_tol = 1e-8;
    int max_iter = 1000;
    int prec = WFQ_PREC_FP64;
    int refine_every = 0;
    double2 *q = nullptr;           // device, n x ncols
    wfq_stats *stats = nullptr;     // host, ncols (may be null)
    // Internal (never set through the C ABI): q already holds an initial guess.
    bool warm = false;
};

// U[d][i] = (D x_d)_i for C <= 4 real direction-major vectors given as float pairs, D
// generated from the coordinates in double-float (matrix-free shifted product).
int d_gemv_df_mf(const wfq_geom *g, int C, const float *xh, const float *xl, double *U, cudaStream_t s);

int solve_gmres(wfq_geom *g, const SolveArgs &a, cudaStream_t s);
int solve_qmr(wfq_geom *g, const SolveArgs &a, cudaStream_t s);
// Shifted GMRES (one real Arnoldi per direction for all frequencies); a.m caps the basis.
// Explicit column lists (a.col_omega / a.col_dir over a.ndir directions) are accepted.
int solve_gmres_shifted(wfq_geom *g, const SolveArgs &a, cudaStream_t s);
// Device bytes a shifted solve of ncols columns over ndir directions allocates (m: basis cap).
size_t shifted_footprint(const wfq_geom *g, int64_t ncols, int ndir, int m);
// FP64 true residual of every column of a (iterate in a.q); columns above a.rel_tol continue
// in block GMRES(m) at a.prec.  iters: Krylov steps already spent per column.  dq: D a.q
// (n x ncols) when the caller has it, else null (computed with double-float products).
int finish_columns(wfq_geom *g, const SolveArgs &a, const std::vector<int> &iters, int m, const double2 *dq,
                   cudaStream_t s);

// Device bytes a block solve of `cc` columns allocates (Krylov basis, FP64 blocks, scratch).
size_t solve_footprint(const wfq_geom *g, int64_t cc, int m, int prec);

// The shift model of a geometry's operator family (z_eval).
inline ShiftModel shift_model(const wfq_geom *g) {
    ShiftModel m{};
    m.op = g->op;
    m.n0 = g->p.n0;
    m.tau = g->p.tau;
    m.eps_out = g->bem.eps_out;
    m.eps_inf = g->bem.eps_inf;
    m.wp = g->bem.omega_p;
    m.gamma = g->bem.gamma;
    return m;
}

}  // namespace wfq
