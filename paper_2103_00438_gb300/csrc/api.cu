// C ABI of libwfq (include/wfq.h): argument checking, handle management, host/device
// staging, dispatch to the kernels.
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.h"

namespace wfq {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};
static std::atomic<int64_t> g_allocs{0};   // device allocations requested by the library

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

bool trace_on() {
    static const bool on = [] {
        const char *e = std::getenv("WFQ_TRACE");
        return e != nullptr && *e != '\0' && std::strcmp(e, "0") != 0;
    }();
    return on;
}

void trace(const char *fmt, ...) {
    if (!trace_on()) return;
    static const auto t0 = std::chrono::steady_clock::now();
    const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::fprintf(stderr, "[wfq %9.3f s] %s\n", t, buf);
    std::fflush(stderr);
}

void set_error(const std::string &msg) { g_last_error = msg; }
const char *get_error() { return g_last_error.c_str(); }

int dalloc(wfq_ctx *ctx, void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    note_alloc();
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                  cudaGetErrorString(e));
        return WFQ_ENOMEM;
    }
    return WFQ_OK;
}

void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

cudaEvent_t KernelTimer::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void KernelTimer::collect() {
    for (int k = 0; k < WFQ_KT_COUNT; ++k) {
        for (size_t q = 0; q < pending[k].size(); ++q) {
            auto &pr = pending[k][q];
            float t = 0.f;
            if (cudaEventSynchronize(pr.second) == cudaSuccess &&
                cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) {
                ms[k] += t;
                launches[k] += 1;
                work[k] += pending_work[k][q];
            } else {
                cudaGetLastError();
            }
            pool.push_back(pr.first);
            pool.push_back(pr.second);
        }
        pending[k].clear();
        pending_work[k].clear();
    }
}

void KernelTimer::reset() {
    collect();
    for (int k = 0; k < WFQ_KT_COUNT; ++k) {
        launches[k] = 0;
        ms[k] = 0.0;
        work[k] = 0.0;
    }
}

KernelTimer::~KernelTimer() {
    for (int k = 0; k < WFQ_KT_COUNT; ++k)
        for (auto &pr : pending[k]) pool.push_back(pr.first), pool.push_back(pr.second);
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

KScope::KScope(wfq_ctx *c, int k, cudaStream_t st, double w) : ctx(c), kind(k), s(st), work(w) {
    if (!ctx->timer.enabled) return;
    std::lock_guard<std::mutex> lk(ctx->timer.mu);
    e0 = ctx->timer.get();
    if (e0) cudaEventRecord(e0, s);
}

KScope::~KScope() {
    if (!e0) return;
    std::lock_guard<std::mutex> lk(ctx->timer.mu);
    cudaEvent_t e1 = ctx->timer.get();
    if (!e1) {
        ctx->timer.pool.push_back(e0);
        return;
    }
    cudaEventRecord(e1, s);
    ctx->timer.pending[kind].emplace_back(e0, e1);
    ctx->timer.pending_work[kind].push_back(work);
}

int check_device_error(wfq_ctx *ctx, cudaStream_t s) {
    int h = 0;
    WFQ_CUDA(cudaMemcpyAsync(&h, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    WFQ_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), s);
        return fail(WFQ_ETIMEOUT, "a bounded device-side wait gave up (code " + std::to_string(h) + ")");
    }
    return WFQ_OK;
}

int device_ptr_on(const void *p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type == cudaMemoryTypeManaged) return 1;
    if (at.type != cudaMemoryTypeDevice) return 0;
    return at.device == device ? 1 : -1;
}

// Synchronous device allocation owned by a geometry.
template <class T>
static int galloc(wfq_geom *g, T **p, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    note_alloc();
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(WFQ_ENOMEM, "geometry allocation of " + std::to_string(bytes) + " bytes failed: " +
                                    cudaGetErrorString(e));
    }
    g->bytes += bytes;
    return WFQ_OK;
}

static void free_geom(wfq_geom *g) {
    void *ptrs[] = {g->xyz, g->atom64, g->atom32, g->atom32p, g->atomdf, g->eta, g->rowptr, g->col,
                    g->val64, g->val32, g->D64, g->Dhi, g->Dlo, g->Dfh, g->Dfl,
                    g->Dsym, g->sym_items, g->sym_item_start, g->elem};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    fmm_free(g->fmm);
    delete g;
}

static bool finite_all(const double *a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

static int check_params(const wfq_params *p) {
    if (!p) return fail(WFQ_EINVAL, "params is NULL");
    const double v[] = {p->eta, p->d_fermi, p->s_fermi, p->r0, p->area, p->n0, p->tau};
    const char *names[] = {"eta", "d_fermi", "s_fermi", "r0", "area", "n0", "tau"};
    for (int k = 0; k < 7; ++k)
        if (!(std::isfinite(v[k]) && v[k] > 0.0)) return fail(WFQ_EINVAL, std::string("parameter ") + names[k] + " must be finite and > 0");
    if (!(p->cutoff_eps >= 0.0 && p->cutoff_eps < 1.0)) return fail(WFQ_EINVAL, "cutoff_eps must be in [0, 1)");
    return WFQ_OK;
}

// Device-side view of a caller array that may live on the host: `dev` is what kernels
// use; for host arrays a staging buffer is allocated and copied in/out.
template <class T>
struct Staged {
    T *dev = nullptr;
    T *host = nullptr;
    size_t count = 0;
    DevBuf<T> buf;
    int in(wfq_ctx *ctx, const T *p, size_t cnt, bool copy, cudaStream_t s) {
        count = cnt;
        const int where = device_ptr_on(p, ctx->device);
        if (where < 0) return fail(WFQ_EINVAL, "a device pointer argument lives on another device than the context's");
        if (where > 0) {
            dev = const_cast<T *>(p);
            return WFQ_OK;
        }
        host = const_cast<T *>(p);
        WFQ_TRY(buf.alloc(ctx, cnt, s));
        dev = buf.ptr;
        if (copy) WFQ_CUDA(cudaMemcpyAsync(dev, p, cnt * sizeof(T), cudaMemcpyHostToDevice, s));
        return WFQ_OK;
    }
    int out(cudaStream_t s) {
        if (host) {
            WFQ_CUDA(cudaMemcpyAsync(host, dev, count * sizeof(T), cudaMemcpyDeviceToHost, s));
            WFQ_CUDA(cudaStreamSynchronize(s));
        }
        return WFQ_OK;
    }
};

// Entered by every C-ABI call that touches the device: makes the context's device current
// and clears a runtime error left pending by earlier calls of the caller's own (cudaGetLastError
// after this library's launches must report only what the launches did).
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetLastError();
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace wfq

using namespace wfq;

extern "C" {

const char *wfq_last_error(void) { return get_error(); }

int64_t wfq_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int wfq_memory_stats(wfq_ctx *ctx, int64_t *out) {
    if (!ctx || !out) return fail(WFQ_EINVAL, "NULL argument");
    out[0] = g_allocs.load(std::memory_order_relaxed);
    const cudaMemPoolAttr attrs[3] = {cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrUsedMemCurrent,
                                      cudaMemPoolAttrUsedMemHigh};
    for (int k = 0; k < 3; ++k) {
        unsigned long long v = 0;
        cudaError_t e = cudaMemPoolGetAttribute(ctx->pool, attrs[k], &v);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(WFQ_ECUDA, std::string("cudaMemPoolGetAttribute: ") + cudaGetErrorString(e));
        }
        out[1 + k] = (int64_t)v;
    }
    return WFQ_OK;
}

int wfq_create(wfq_ctx **out, int device) {
    if (!out) return fail(WFQ_EINVAL, "ctx out-pointer is NULL");
    *out = nullptr;
    int count = 0;
    WFQ_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(WFQ_EINVAL, "no such CUDA device");
    DeviceGuard dg(device);
    cudaDeviceProp prop;
    WFQ_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10) return fail(WFQ_EUNSUPPORTED, "libwfq is built for sm_103a (Blackwell) devices");
    auto *ctx = new wfq_ctx;
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    cudaMemPoolProps pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    cudaError_t e = cudaMemPoolCreate(&ctx->pool, &pp);
    if (e != cudaSuccess) {
        delete ctx;
        return fail(WFQ_ECUDA, std::string("cudaMemPoolCreate: ") + cudaGetErrorString(e));
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    note_alloc();
    e = cudaMalloc(&ctx->dev_err, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->dev_err, 0, 256);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(ctx->pool);
        delete ctx;
        return fail(WFQ_ECUDA, std::string("context flag allocation: ") + cudaGetErrorString(e));
    }
    *out = ctx;
    return WFQ_OK;
}

int wfq_destroy(wfq_ctx *ctx) {
    if (!ctx) return WFQ_OK;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->dev_err) cudaFree(ctx->dev_err);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    delete ctx;
    return WFQ_OK;
}

int wfq_profile(wfq_ctx *ctx, int enable) {
    if (!ctx) return fail(WFQ_EINVAL, "NULL context");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->timer.mu);
    if (enable) ctx->timer.reset();
    ctx->timer.enabled = enable != 0;
    return WFQ_OK;
}

int wfq_profile_read(wfq_ctx *ctx, int kind, int64_t *launches, double *total_ms, double *work) {
    if (!ctx) return fail(WFQ_EINVAL, "NULL context");
    if (kind < 0 || kind >= WFQ_KT_COUNT) return fail(WFQ_EINVAL, "unknown kernel class");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->timer.mu);
    ctx->timer.collect();
    if (launches) *launches = ctx->timer.launches[kind];
    if (total_ms) *total_ms = ctx->timer.ms[kind];
    if (work) *work = ctx->timer.work[kind];
    return WFQ_OK;
}

int wfq_build_geometry(wfq_ctx *ctx, int64_t n, const double *xyz, const double *eta, const wfq_params *p,
                       uint32_t store, wfq_geom **out) {
    if (!ctx || !out) return fail(WFQ_EINVAL, "NULL context or out-pointer");
    *out = nullptr;
    if (n < 1) return fail(WFQ_EINVAL, "n must be >= 1");
    if (!xyz) return fail(WFQ_EINVAL, "xyz is NULL");
    if (store & ~(WFQ_STORE_FP64 | WFQ_STORE_BF16X2 | WFQ_STORE_F32X2 | WFQ_STORE_F32X2_SYM))
        return fail(WFQ_EINVAL, "unknown storage flag");
    WFQ_TRY(check_params(p));
    if (!finite_all(xyz, 3 * n)) return fail(WFQ_EINVAL, "xyz has a non-finite entry");
    std::vector<double> eta_h(n, p->eta);
    if (eta) {
        for (int64_t i = 0; i < n; ++i) {
            if (!(std::isfinite(eta[i]) && eta[i] > 0.0)) return fail(WFQ_EINVAL, "eta entries must be finite and > 0");
            eta_h[i] = eta[i];
        }
    }
    if (n > INT32_MAX) return fail(WFQ_EINVAL, "n exceeds 2^31 - 1");
    DeviceGuard dg(ctx->device);

    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    std::vector<double> val;
    WFQ_TRY(build_kbar_csr(n, xyz, *p, rowptr, col, val));

    auto *g = new wfq_geom;
    g->ctx = ctx;
    g->n = n;
    g->npad = round_up(n, kTilePad);
    g->ldf = round_up(n, 128);
    g->p = *p;
    g->store = store;
    g->nnz = rowptr[n];
    int rc = WFQ_OK;
    auto bail = [&](int code) {
        free_geom(g);
        return code;
    };
    std::vector<atom64_t> a64(n);
    std::vector<float4> a32(g->npad);
    const double wfac = std::sqrt(2.0 / M_PI);  // Eq. 4
    for (int64_t i = 0; i < n; ++i) {
        double w = wfac / eta_h[i];
        a64[i] = atom64_t{xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], w};
        a32[i] = make_float4((float)xyz[3 * i], (float)xyz[3 * i + 1], (float)xyz[3 * i + 2], (float)w);
    }
    for (int64_t i = n; i < g->npad; ++i) a32[i] = make_float4(1e30f, 1e30f, 1e30f, 1.0f);
    std::vector<float4> adf(2 * n);
    auto split = [](double v, float &h, float &l) {
        h = (float)v;
        l = (float)(v - (double)h);
    };
    for (int64_t i = 0; i < n; ++i) {
        float xh, xl, yh, yl, zh, zl;
        split(xyz[3 * i], xh, xl);
        split(xyz[3 * i + 1], yh, yl);
        split(xyz[3 * i + 2], zh, zl);
        adf[2 * i] = make_float4(xh, xl, yh, yl);
        adf[2 * i + 1] = make_float4(zh, zl, (float)(wfac / eta_h[i]), 0.0f);
    }
    std::vector<float> val32(val.begin(), val.end());

    if ((rc = galloc(g, &g->xyz, 3 * n))) return bail(rc);
    if ((rc = galloc(g, &g->atom64, n))) return bail(rc);
    if ((rc = galloc(g, &g->atom32, g->npad))) return bail(rc);
    if ((rc = galloc(g, &g->atom32p, g->npad))) return bail(rc);
    if ((rc = galloc(g, &g->atomdf, 2 * n))) return bail(rc);
    if ((rc = galloc(g, &g->eta, n))) return bail(rc);
    if ((rc = galloc(g, &g->rowptr, n + 1))) return bail(rc);
    if ((rc = galloc(g, &g->col, g->nnz))) return bail(rc);
    if ((rc = galloc(g, &g->val64, g->nnz))) return bail(rc);
    if ((rc = galloc(g, &g->val32, g->nnz))) return bail(rc);
    if (store & WFQ_STORE_FP64)
        if ((rc = galloc(g, &g->D64, (size_t)n * n))) return bail(rc);
    if (store & WFQ_STORE_BF16X2) {
        if ((rc = galloc(g, &g->Dhi, (size_t)g->npad * g->npad))) return bail(rc);
        if ((rc = galloc(g, &g->Dlo, (size_t)g->npad * g->npad))) return bail(rc);
    }
    if (store & WFQ_STORE_F32X2) {
        if ((rc = galloc(g, &g->Dfh, (size_t)n * g->ldf))) return bail(rc);
        if ((rc = galloc(g, &g->Dfl, (size_t)n * g->ldf))) return bail(rc);
    }
    std::vector<SymItem> sym_items;
    std::vector<int> sym_start;
    if (store & WFQ_STORE_F32X2_SYM) {
        // work items of the symmetric product: each tile row split into runs of at most
        // kSymChunk tiles (balances the triangle's long and short rows)
        const int64_t T = (n + kSymTile - 1) / kSymTile;
        const int kSymChunk = 16;
        g->sym_nt = T;
        for (int64_t I = 0; I < T; ++I) {
            sym_start.push_back((int)sym_items.size());
            for (int64_t J0 = I; J0 < T; J0 += kSymChunk)
                sym_items.push_back(SymItem{(int)I, (int)J0, (int)std::min<int64_t>(J0 + kSymChunk, T), 0});
        }
        sym_start.push_back((int)sym_items.size());
        g->sym_nitems = (int64_t)sym_items.size();
        if ((rc = galloc(g, &g->Dsym, (size_t)(T * (T + 1) / 2) * 2 * kSymTile * kSymTile))) return bail(rc);
        if ((rc = galloc(g, &g->sym_items, sym_items.size()))) return bail(rc);
        if ((rc = galloc(g, &g->sym_item_start, sym_start.size()))) return bail(rc);
    }
    auto up = [&](void *dst, const void *src, size_t bytes) -> int {
        if (bytes == 0) return WFQ_OK;
        cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(WFQ_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
        return WFQ_OK;
    };
    if ((rc = up(g->xyz, xyz, sizeof(double) * 3 * n))) return bail(rc);
    if ((rc = up(g->atom64, a64.data(), sizeof(atom64_t) * n))) return bail(rc);
    if ((rc = up(g->atom32, a32.data(), sizeof(float4) * g->npad))) return bail(rc);
    {
        std::vector<float4> a32p(g->npad);   // npad is a multiple of 128: whole pairs
        for (int64_t k = 0; k < g->npad; k += 2) {
            const float4 a = a32[k], b = a32[k + 1];
            a32p[k] = make_float4(a.x, b.x, a.y, b.y);
            a32p[k + 1] = make_float4(a.z, b.z, a.w, b.w);
        }
        if ((rc = up(g->atom32p, a32p.data(), sizeof(float4) * g->npad))) return bail(rc);
    }
    if ((rc = up(g->atomdf, adf.data(), sizeof(float4) * 2 * n))) return bail(rc);
    if ((rc = up(g->eta, eta_h.data(), sizeof(double) * n))) return bail(rc);
    if ((rc = up(g->rowptr, rowptr.data(), sizeof(int64_t) * (n + 1)))) return bail(rc);
    if ((rc = up(g->col, col.data(), sizeof(int32_t) * g->nnz))) return bail(rc);
    if ((rc = up(g->val64, val.data(), sizeof(double) * g->nnz))) return bail(rc);
    if ((rc = up(g->val32, val32.data(), sizeof(float) * g->nnz))) return bail(rc);
    if (!sym_items.empty()) {
        if ((rc = up(g->sym_items, sym_items.data(), sizeof(SymItem) * sym_items.size()))) return bail(rc);
        if ((rc = up(g->sym_item_start, sym_start.data(), sizeof(int) * sym_start.size()))) return bail(rc);
    }
    if ((rc = launch_build_d(g, nullptr))) return bail(rc);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bail(fail(WFQ_ECUDA, std::string("D build: ") + cudaGetErrorString(e)));
    *out = g;
    return WFQ_OK;
}

int wfq_build_bem_geometry(wfq_ctx *ctx, int64_t n, const double *xyz, const double *normal, const double *area,
                           const double *curvature, const wfq_bem_params *p, uint32_t store, wfq_geom **out) {
    if (!ctx || !out) return fail(WFQ_EINVAL, "NULL context or out-pointer");
    *out = nullptr;
    if (n < 1) return fail(WFQ_EINVAL, "n must be >= 1");
    if (n > INT32_MAX) return fail(WFQ_EINVAL, "n exceeds 2^31 - 1");
    if (!xyz || !normal || !area || !p) return fail(WFQ_EINVAL, "xyz, normal, area or params is NULL");
    if (store & ~(WFQ_STORE_FP64 | WFQ_STORE_BF16X2 | WFQ_STORE_F32X2 | WFQ_STORE_F32X2_SYM))
        return fail(WFQ_EINVAL, "unknown storage flag");
    if (!(store & WFQ_STORE_FP64)) return fail(WFQ_EINVAL, "the BEM operator needs WFQ_STORE_FP64");
    if (store & WFQ_STORE_F32X2_SYM) return fail(WFQ_EINVAL, "the BEM operator is not symmetric: no WFQ_STORE_F32X2_SYM");
    if (!(std::isfinite(p->eps_out) && p->eps_out > 0.0 && std::isfinite(p->eps_inf) && p->eps_inf > 0.0 &&
          std::isfinite(p->omega_p) && p->omega_p > 0.0 && std::isfinite(p->gamma) && p->gamma >= 0.0))
        return fail(WFQ_EINVAL, "BEM parameters: eps_out, eps_inf, omega_p must be finite and > 0, gamma finite and >= 0");
    if (!finite_all(xyz, 3 * n) || !finite_all(normal, 3 * n) || !finite_all(area, n) ||
        (curvature && !finite_all(curvature, n)))
        return fail(WFQ_EINVAL, "non-finite position, normal, area or curvature");
    std::vector<elem64_t> el(n);
    for (int64_t i = 0; i < n; ++i) {
        const double nx = normal[3 * i], ny = normal[3 * i + 1], nz = normal[3 * i + 2];
        if (std::fabs(std::sqrt(nx * nx + ny * ny + nz * nz) - 1.0) > 1e-6)
            return fail(WFQ_EINVAL, "normal " + std::to_string(i) + " is not a unit vector");
        if (!(area[i] > 0.0)) return fail(WFQ_EINVAL, "element areas must be > 0");
        const double H = curvature ? curvature[i] : 0.0;
        // self coefficient: Eq. 22's principal value over the element itself, a disk of the
        // element's area (radius rho = sqrt(a / pi)) on a surface of mean curvature H, where
        // n . (r_i - r') / |r_i - r'|^3 is about H / (2 s) at distance s: pi H rho in total.
        // The charge form (row scaled by a_i, unknown a_i sigma_i) leaves it unchanged.
        el[i] = elem64_t{xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], nx, ny, nz, area[i],
                         H * std::sqrt(M_PI * area[i])};
    }
    DeviceGuard dg(ctx->device);
    auto *g = new wfq_geom;
    g->ctx = ctx;
    g->op = OP_BEM;
    g->n = n;
    g->npad = round_up(n, kTilePad);
    g->ldf = round_up(n, 128);
    g->bem = *p;
    g->store = store;
    g->nnz = 0;
    int rc = WFQ_OK;
    auto bail = [&](int code) {
        free_geom(g);
        return code;
    };
    if ((rc = galloc(g, &g->xyz, 3 * n))) return bail(rc);
    if ((rc = galloc(g, &g->elem, n))) return bail(rc);
    if ((rc = galloc(g, &g->rowptr, n + 1))) return bail(rc);   // empty sparse term
    if ((rc = galloc(g, &g->D64, (size_t)n * n))) return bail(rc);
    if (store & WFQ_STORE_BF16X2) {
        if ((rc = galloc(g, &g->Dhi, (size_t)g->npad * g->npad))) return bail(rc);
        if ((rc = galloc(g, &g->Dlo, (size_t)g->npad * g->npad))) return bail(rc);
    }
    if (store & WFQ_STORE_F32X2) {
        if ((rc = galloc(g, &g->Dfh, (size_t)n * g->ldf))) return bail(rc);
        if ((rc = galloc(g, &g->Dfl, (size_t)n * g->ldf))) return bail(rc);
    }
    // device flag of the build kernel: two elements closer than 1e-8 bohr (freed below)
    int *close = nullptr;
    note_alloc();
    cudaError_t e = cudaMalloc(&close, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(WFQ_ENOMEM, std::string("BEM build flag: ") + cudaGetErrorString(e)));
    }
    auto done = [&](int code) {
        cudaFree(close);
        return code == WFQ_OK ? WFQ_OK : bail(code);
    };
    e = cudaMemcpy(g->xyz, xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->elem, el.data(), sizeof(elem64_t) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(g->rowptr, 0, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMemset(close, 0, sizeof(int));
    if (e != cudaSuccess) return done(fail(WFQ_ECUDA, std::string("upload: ") + cudaGetErrorString(e)));
    if ((rc = launch_build_bem(g, close, nullptr))) return done(rc);
    int close_h = 0;
    e = cudaMemcpy(&close_h, close, sizeof(int), cudaMemcpyDeviceToHost);   // synchronises the build
    if (e != cudaSuccess) return done(fail(WFQ_ECUDA, std::string("BEM build: ") + cudaGetErrorString(e)));
    if (close_h) return done(fail(WFQ_EINVAL, "two surface elements closer than 1e-8 bohr"));
    done(WFQ_OK);
    *out = g;
    return WFQ_OK;
}

int wfq_free_geometry(wfq_geom *g) {
    if (!g) return WFQ_OK;
    DeviceGuard dg(g->ctx->device);
    cudaDeviceSynchronize();
    free_geom(g);
    return WFQ_OK;
}

int wfq_geometry_info(const wfq_geom *g, int64_t *n, int64_t *nnz, int64_t *device_bytes) {
    if (!g) return fail(WFQ_EINVAL, "geometry is NULL");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (device_bytes) *device_bytes = (int64_t)g->bytes;
    return WFQ_OK;
}

int wfq_apply(wfq_geom *g, int64_t ncplx, const double *omega, const void *x, void *y, int prec, void *stream) {
    if (!g || !omega || !x || !y) return fail(WFQ_EINVAL, "NULL argument");
    if (ncplx < 1) return fail(WFQ_EINVAL, "ncplx must be >= 1");
    if (prec != WFQ_PREC_FP64 && prec != WFQ_PREC_MIXED && prec != WFQ_PREC_DF && prec != WFQ_PREC_FMM)
        return fail(WFQ_EINVAL, "unknown precision");
    if (prec == WFQ_PREC_FMM && !g->fmm)
        return fail(WFQ_EUNSUPPORTED, "WFQ_PREC_FMM needs wfq_fmm_build on this geometry first");
    if (prec == WFQ_PREC_FMM && ncplx > 256)
        return fail(WFQ_EINVAL, "WFQ_PREC_FMM applies at most 256 complex columns per call");
    if (!finite_all(omega, ncplx)) return fail(WFQ_EINVAL, "omega has a non-finite entry");
    DeviceGuard dg(g->ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = g->n, nc = n * ncplx;
    std::vector<double2> zh(ncplx);
    if (g->op == OP_BEM && prec == WFQ_PREC_MIXED && !g->Dhi)
        return fail(WFQ_EUNSUPPORTED, "the mixed apply of a BEM geometry needs WFQ_STORE_BF16X2");
    const ShiftModel zm = shift_model(g);
    for (int64_t c = 0; c < ncplx; ++c) {
        zh[c] = z_eval(zm, omega[c]);
        if (!(std::isfinite(zh[c].x) && std::isfinite(zh[c].y)))
            return fail(WFQ_EINVAL, "z(omega) is not finite (BEM: omega = 0 or eps_in = eps_out)");
    }
    DevBuf<double2> z;
    WFQ_TRY(z.alloc(g->ctx, ncplx, s));
    WFQ_CUDA(cudaMemcpyAsync(z.ptr, zh.data(), sizeof(double2) * ncplx, cudaMemcpyHostToDevice, s));
    if (prec == WFQ_PREC_FP64 || prec == WFQ_PREC_DF) {
        Staged<double2> X, Y;
        WFQ_TRY(X.in(g->ctx, static_cast<const double2 *>(x), nc, true, s));
        WFQ_TRY(Y.in(g->ctx, static_cast<double2 *>(y), nc, false, s));
        DevBuf<double2> U;
        WFQ_TRY(U.alloc(g->ctx, nc, s));
        if (prec == WFQ_PREC_DF)
            WFQ_TRY(d_apply_df(g, ncplx, X.dev, U.ptr, s));
        else
            WFQ_TRY(d_apply_fp64(g, ncplx, X.dev, U.ptr, s));
        WFQ_TRY(sparse_shift_fp64(g, ncplx, U.ptr, X.dev, z.ptr, Y.dev, s));
        WFQ_TRY(Y.out(s));
    } else {
        Staged<float2> X, Y;
        WFQ_TRY(X.in(g->ctx, static_cast<const float2 *>(x), nc, true, s));
        WFQ_TRY(Y.in(g->ctx, static_cast<float2 *>(y), nc, false, s));
        DevBuf<float2> U;
        DevBuf<unsigned char> scratch;
        WFQ_TRY(U.alloc(g->ctx, nc, s));
        if (prec == WFQ_PREC_FMM) {
            WFQ_TRY(d_apply_fmm(g, ncplx, X.dev, U.ptr, s));
        } else {
            WFQ_TRY(scratch.alloc(g->ctx, mixed_scratch_bytes(g, ncplx), s));
            WFQ_TRY(d_apply_mixed(g, ncplx, X.dev, U.ptr, scratch.ptr, s));
        }
        WFQ_TRY(sparse_shift_fp32(g, ncplx, U.ptr, X.dev, z.ptr, Y.dev, s));
        WFQ_TRY(Y.out(s));
    }
    WFQ_CUDA(cudaGetLastError());
    return WFQ_OK;
}

int wfq_fmm_build(wfq_geom *g, int order) {
    if (!g) return fail(WFQ_EINVAL, "geometry is NULL");
    if (order < 2 || order > 16) return fail(WFQ_EINVAL, "FMM order must be in 2..16");
    if (g->op != OP_WFQ) return fail(WFQ_EUNSUPPORTED, "the FMM product takes omega-FQ geometries only");
    DeviceGuard dg(g->ctx->device);
    WFQ_CUDA(cudaDeviceSynchronize());
    Fmm *f = nullptr;
    WFQ_TRY(fmm_build(g, order, &f));
    if (g->fmm) {
        g->bytes -= fmm_bytes(g->fmm);
        fmm_free(g->fmm);
    }
    g->fmm = f;
    g->bytes += fmm_bytes(f);
    return WFQ_OK;
}

int wfq_fmm_info(const wfq_geom *g, int64_t *out) {
    if (!g || !out) return fail(WFQ_EINVAL, "NULL argument");
    if (!g->fmm) return fail(WFQ_EUNSUPPORTED, "wfq_fmm_build has not been called on this geometry");
    fmm_info(g->fmm, out);
    return WFQ_OK;
}

int wfq_rhs(wfq_geom *g, int ndir, const double *dirs, double E0, double *R, void *stream) {
    if (!g || !dirs || !R) return fail(WFQ_EINVAL, "NULL argument");
    if (ndir < 1) return fail(WFQ_EINVAL, "ndir must be >= 1");
    if (!finite_all(dirs, 3 * ndir) || !std::isfinite(E0)) return fail(WFQ_EINVAL, "non-finite direction or E0");
    DeviceGuard dg(g->ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevBuf<double> d;
    WFQ_TRY(d.alloc(g->ctx, 3 * ndir, s));
    WFQ_CUDA(cudaMemcpyAsync(d.ptr, dirs, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, s));
    Staged<double> Rs;
    WFQ_TRY(Rs.in(g->ctx, R, (size_t)g->n * ndir, false, s));
    WFQ_TRY(launch_rhs(g, ndir, d.ptr, E0, Rs.dev, s));
    WFQ_TRY(Rs.out(s));
    return WFQ_OK;
}

enum Solver { SOLVE_GMRES, SOLVE_QMR, SOLVE_SHIFTED };

static int solve_common(Solver kind, wfq_geom *g, int64_t nfreq, const double *omega, int ndir, const double *dirs,
                        double E0, int m, double rel_tol, int max_iter, int prec, int refine_every, double *q,
                        wfq_stats *stats, void *stream) {
    if (!g || !omega || !dirs || !q) return fail(WFQ_EINVAL, "NULL argument");
    if (nfreq < 1 || ndir < 1) return fail(WFQ_EINVAL, "nfreq and ndir must be >= 1");
    if (m < 0 || max_iter < 1 || refine_every < 0) return fail(WFQ_EINVAL, "m, max_iter or refine_every out of range");
    if (!(rel_tol > 0.0 && rel_tol < 1.0)) return fail(WFQ_EINVAL, "rel_tol must be in (0, 1)");
    if (prec != WFQ_PREC_FP64 && prec != WFQ_PREC_MIXED) return fail(WFQ_EINVAL, "unknown precision");
    if (!finite_all(omega, nfreq) || !finite_all(dirs, 3 * (int64_t)ndir) || !std::isfinite(E0) || E0 == 0.0)
        return fail(WFQ_EINVAL, "non-finite omega / direction or E0 = 0");
    for (int64_t f = 0; f < nfreq; ++f)
        if (omega[f] == 0.0) return fail(WFQ_ESINGULAR, "omega = 0: z(0) = 0 and A is singular");
    if (g->op == OP_BEM) {
        if (kind == SOLVE_QMR)
            return fail(WFQ_EUNSUPPORTED, "J-symmetric QMR needs A = (Kbar - P) D with D symmetric; "
                                          "the BEM operator has no such factor");
        if (prec == WFQ_PREC_MIXED && !g->Dhi)
            return fail(WFQ_EUNSUPPORTED, "WFQ_PREC_MIXED on a BEM geometry needs WFQ_STORE_BF16X2");
        const ShiftModel zm = shift_model(g);
        for (int64_t f = 0; f < nfreq; ++f) {
            const double2 z = z_eval(zm, omega[f]);
            if (!(std::isfinite(z.x) && std::isfinite(z.y)))
                return fail(WFQ_EINVAL, "eps_in(omega) = eps_out: Lambda(omega) is infinite");
        }
    }
    DeviceGuard dg(g->ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t cc = nfreq * ndir;
    Staged<double2> Q;
    WFQ_TRY(Q.in(g->ctx, reinterpret_cast<double2 *>(q), (size_t)g->n * cc, false, s));
    SolveArgs a;
    a.nfreq = nfreq;
    a.omega = omega;
    a.ndir = ndir;
    a.dirs = dirs;
    a.E0 = E0;
    a.m = m;
    a.rel_tol = rel_tol;
    a.max_iter = max_iter;
    a.prec = prec;
    a.refine_every = refine_every;
    a.q = Q.dev;
    a.stats = stats;
    int rc = kind == SOLVE_QMR ? solve_qmr(g, a, s)
             : kind == SOLVE_SHIFTED ? solve_gmres_shifted(g, a, s)
                                     : solve_gmres(g, a, s);
    if (rc != WFQ_OK && rc != WFQ_ENOCONV && rc != WFQ_EBREAKDOWN) return rc;
    WFQ_TRY(Q.out(s));
    WFQ_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int wfq_solve_gmres(wfq_geom *g, int64_t nfreq, const double *omega, int ndir, const double *dirs, double E0, int m,
                    double rel_tol, int max_iter, int prec, double *q, wfq_stats *stats, void *stream) {
    return solve_common(SOLVE_GMRES, g, nfreq, omega, ndir, dirs, E0, m, rel_tol, max_iter, prec, 0, q, stats,
                        stream);
}

int wfq_solve_gmres_shifted(wfq_geom *g, int64_t nfreq, const double *omega, int ndir, const double *dirs,
                            double E0, int m_max, double rel_tol, int max_iter, int prec, double *q,
                            wfq_stats *stats, void *stream) {
    return solve_common(SOLVE_SHIFTED, g, nfreq, omega, ndir, dirs, E0, m_max, rel_tol, max_iter, prec, 0, q, stats,
                        stream);
}

int wfq_solve_qmr(wfq_geom *g, int64_t nfreq, const double *omega, int ndir, const double *dirs, double E0,
                  double rel_tol, int max_iter, int prec, int refine_every, double *q, wfq_stats *stats,
                  void *stream) {
    return solve_common(SOLVE_QMR, g, nfreq, omega, ndir, dirs, E0, 0, rel_tol, max_iter, prec, refine_every, q, stats,
                        stream);
}

int wfq_polarizability(wfq_geom *g, int64_t ncols, const double *q, double E0, double *alpha, void *stream) {
    if (!g || !q || !alpha) return fail(WFQ_EINVAL, "NULL argument");
    if (ncols < 1) return fail(WFQ_EINVAL, "ncols must be >= 1");
    if (!std::isfinite(E0) || E0 == 0.0) return fail(WFQ_EINVAL, "E0 must be finite and non-zero");
    DeviceGuard dg(g->ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Staged<double2> Q;
    WFQ_TRY(Q.in(g->ctx, reinterpret_cast<const double2 *>(q), (size_t)g->n * ncols, true, s));
    Staged<double2> A;
    WFQ_TRY(A.in(g->ctx, reinterpret_cast<double2 *>(alpha), (size_t)ncols * 3, false, s));
    WFQ_TRY(launch_polarizability(g, ncols, Q.dev, E0, A.dev, s));
    WFQ_TRY(A.out(s));
    WFQ_CUDA(cudaStreamSynchronize(s));
    return WFQ_OK;
}

int wfq_cross_section(wfq_geom *g, int64_t nfreq, const double *omega, int ndir, const double *dirs,
                      double E0, const double *q, double *sigma, double *sigma_iso, void *stream) {
    if (!g || !omega || !dirs || !q || !sigma) return fail(WFQ_EINVAL, "NULL argument");
    if (nfreq < 1 || ndir < 1) return fail(WFQ_EINVAL, "nfreq and ndir must be >= 1");
    if (!std::isfinite(E0) || E0 == 0.0) return fail(WFQ_EINVAL, "E0 must be finite and non-zero");
    for (int64_t f = 0; f < nfreq; ++f)
        if (!std::isfinite(omega[f])) return fail(WFQ_EINVAL, "omega has a non-finite entry");
    for (int d = 0; d < ndir; ++d) {
        const double *k = dirs + 3 * d;
        const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        if (!(std::isfinite(kk) && kk > 0.0)) return fail(WFQ_EINVAL, "each direction must be finite and non-zero");
    }
    DeviceGuard dg(g->ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t ncols = nfreq * (int64_t)ndir;
    Staged<double2> Q;
    WFQ_TRY(Q.in(g->ctx, reinterpret_cast<const double2 *>(q), (size_t)g->n * ncols, true, s));
    DevBuf<double> par;   // omega, then dirs
    WFQ_TRY(par.alloc(g->ctx, (size_t)nfreq + 3 * (size_t)ndir, s));
    WFQ_CUDA(cudaMemcpyAsync(par.ptr, omega, sizeof(double) * nfreq, cudaMemcpyHostToDevice, s));
    WFQ_CUDA(cudaMemcpyAsync(par.ptr + nfreq, dirs, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, s));
    Staged<double> SG, SI;
    WFQ_TRY(SG.in(g->ctx, sigma, (size_t)ncols, false, s));
    if (sigma_iso) WFQ_TRY(SI.in(g->ctx, sigma_iso, (size_t)nfreq, false, s));
    WFQ_TRY(launch_cross_section(g, nfreq, ndir, par.ptr, par.ptr + nfreq, Q.dev, E0, SG.dev,
                                 sigma_iso ? SI.dev : nullptr, s));
    WFQ_TRY(SG.out(s));
    if (sigma_iso) WFQ_TRY(SI.out(s));
    WFQ_CUDA(cudaStreamSynchronize(s));
    return WFQ_OK;
}

}  // extern "C"
