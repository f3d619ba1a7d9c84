// wfq_apply_mixed_noalloc: the mixed-precision operator apply (the same kernels as
// wfq_apply with WFQ_PREC_MIXED) for callers that cannot allocate device memory --
// for example code running inside a pre-sized memory arena or a host callback where
// cudaMalloc is forbidden or would synchronise the device.  Its scratch (the bf16 hi/lo
// planes of x, the product u = D x and the shifts z) lives in one static device array
// instead of coming from the allocator, and the frequencies reach the device as a
// kernel argument instead of a copy.
#include <atomic>
#include <cmath>
#include <mutex>

#include "common.h"

namespace wfq {

// Size of the static scratch array; every device that loads the library holds it
// until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device with that
// device current (in host code the symbol is only a host-side stand-in).
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[kMaxDevices] = {};

static int noalloc_scratch(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return fail(WFQ_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return fail(WFQ_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        }
        g_noalloc_addr[device] = p;
    }
    *out = g_noalloc_addr[device];
    return WFQ_OK;
}

// The column frequencies travel as a kernel argument (no host-to-device copy of a
// caller's array); one thread per column writes z(omega_c) into the scratch slot, with
// the shift of the geometry's operator (z_eval: Eq. 12 for omega-FQ).
constexpr int64_t kNoAllocMaxCols = 1024;
struct NoallocOmega {
    double w[kNoAllocMaxCols];
};

__global__ void k_noalloc_z(int64_t ncplx, ShiftModel m, NoallocOmega om, double2 *__restrict__ z) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncplx) return;
    z[c] = z_eval(m, om.w[c]);
}

static inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace wfq

using namespace wfq;

extern "C" int wfq_apply_mixed_noalloc(wfq_geom *g, int64_t ncplx, const double *omega, const void *x, void *y,
                                       void *stream) {
    if (!g || !omega || !x || !y) return fail(WFQ_EINVAL, "NULL argument");
    if (ncplx < 1) return fail(WFQ_EINVAL, "ncplx must be >= 1");
    if (ncplx > kNoAllocMaxCols)
        return fail(WFQ_EINVAL, "wfq_apply_mixed_noalloc takes at most " + std::to_string(kNoAllocMaxCols) +
                                    " columns per call (its frequencies travel as a kernel argument); use wfq_apply");
    if (!g->Dhi) return fail(WFQ_EUNSUPPORTED, "the mixed apply needs WFQ_STORE_BF16X2");
    if (g->op != OP_WFQ) return fail(WFQ_EUNSUPPORTED, "wfq_apply_mixed_noalloc takes omega-FQ geometries only");
    for (int64_t c = 0; c < ncplx; ++c)
        if (!std::isfinite(omega[c])) return fail(WFQ_EINVAL, "omega has a non-finite entry");
    const int64_t n = g->n;
    const size_t z_bytes = align256(sizeof(double2) * (size_t)ncplx);
    const size_t u_bytes = align256(sizeof(float2) * (size_t)n * (size_t)ncplx);
    const size_t plane_bytes = mixed_scratch_bytes(g, ncplx);
    const size_t need = z_bytes + u_bytes + plane_bytes;
    if (need > kNoAllocScratchBytes)
        return fail(WFQ_EINVAL, "wfq_apply_mixed_noalloc: this size needs " + std::to_string(need) +
                                    " bytes of scratch, more than the static " +
                                    std::to_string(kNoAllocScratchBytes) + "-byte array; use wfq_apply");
    cudaGetLastError();   // an error left pending by the caller's earlier calls is not this call's
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->ctx->device) WFQ_CUDA(cudaSetDevice(g->ctx->device));
    int rc = WFQ_OK;
    do {
        if (device_ptr_on(x, g->ctx->device) <= 0 || device_ptr_on(y, g->ctx->device) <= 0) {
            rc = fail(WFQ_EINVAL, "wfq_apply_mixed_noalloc takes device pointers of the context's device for x and y");
            break;
        }
        void *base = nullptr;
        if ((rc = noalloc_scratch(g->ctx->device, &base)) != WFQ_OK) break;
        unsigned char *b = static_cast<unsigned char *>(base);
        double2 *z = reinterpret_cast<double2 *>(b);
        float2 *u = reinterpret_cast<float2 *>(b + z_bytes);
        void *planes = b + z_bytes + u_bytes;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        NoallocOmega om;
        for (int64_t c = 0; c < ncplx; ++c) om.w[c] = omega[c];
        k_noalloc_z<<<(unsigned)((ncplx + 127) / 128), 128, 0, s>>>(ncplx, shift_model(g), om, z);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = fail(WFQ_ECUDA, std::string("z kernel: ") + cudaGetErrorString(e));
            break;
        }
        if ((rc = d_apply_mixed(g, ncplx, static_cast<const float2 *>(x), u, planes, s)) != WFQ_OK) break;
        rc = sparse_shift_fp32(g, ncplx, u, static_cast<const float2 *>(x), z, static_cast<float2 *>(y), s);
    } while (0);
    if (prev >= 0 && prev != g->ctx->device) cudaSetDevice(prev);
    return rc;
}
