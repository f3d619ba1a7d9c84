// Tensor-core GEMM for the dense product of the mixed operator (sm_103a):
//
//     U[i][c] = sum_k  Dhi[i][k] Xhi[c][k] + Dhi[i][k] Xlo[c][k] + Dlo[i][k] Xhi[c][k]
//
// D ~= Dhi + Dlo and X ~= Xhi + Xlo are bf16 splits (16 significant bits); the three
// products are accumulated in FP32 in tensor memory.  Both operands are K-major (the
// atom index k is contiguous in memory), so this is one "TN" GEMM with M = rows of D,
// N = real columns of the block, K = atoms.
//
// Structure (one CTA per SM, persistent):
//   warp 0   : TMEM allocation; one lane issues the TMA loads of every pipeline stage
//              (Dhi, Dlo tiles of 128 x 32 and Xhi, Xlo tiles of cpad x 32, 64-byte
//              swizzle) and signals a full-barrier with the byte count.
//   warp 1   : one lane issues tcgen05.mma (M = 128, N <= 256 per instruction, K = 16)
//              for the three products and commits each stage back to its empty-barrier.
//   warps 2-5: epilogue -- tcgen05.ld of the 128 x cpad FP32 accumulator, plain stores
//              for tiles the CTA owns whole, FP32 atomics for tiles shared with one
//              neighbour CTA (stream-K split of the K range).
// Work split: the (row tile, k block) units are cut into equal contiguous ranges, one per
// CTA.  With at least one full tile per CTA a tile is shared by at most two CTAs, so the
// two atomic adds onto a zeroed U commute and the result does not depend on timing.
// Every barrier wait is bounded (%globaltimer): on timeout the kernel records an error
// code, stops issuing work, waits (bounded) for what it already issued, frees TMEM and
// returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>

#include "tma_util.cuh"

namespace wfq {
namespace tc {

constexpr int BM = 128;            // rows of D per tile = MMA M
constexpr int BK = 32;             // atoms per pipeline stage: one 64-byte swizzle row
constexpr int ROWB = BK * 2;       // bytes per tile row in shared memory
constexpr int NUM_THREADS = 192;
constexpr int MAX_STAGES = 8;
constexpr uint32_t A_BYTES = BM * ROWB;   // 8 KiB per D plane per stage

struct Params {
    int64_t n;         // valid rows of U
    int64_t ldu;       // row stride of U (floats)
    int64_t ncols;     // valid columns of U in this launch
    int64_t units;     // mtiles * kblocks
    int kblocks;       // npad / BK
    int cpad;          // accumulator columns (multiple of 32, <= 512)
    int nsplit;        // MMA instructions across N
    int nchunk;        // columns per MMA instruction (multiple of 16, <= 256)
    int stages;
    int tmem_cols;     // power of two >= cpad
    uint32_t stage_bytes;
    uint32_t b_bytes;  // cpad * ROWB
    float *U;
    int *err;
    unsigned long long timeout_ns;
};

// Bounded wait for the completion of the phase with the given parity.  Returns false
// (after recording `code` and raising the CTA abort flag) on timeout or if another
// role already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const Params &p, int code,
                                          volatile int *abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 127u) == 0u) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > p.timeout_ns) {
                atomicCAS(p.err, 0, code);
                *abort_flag = 1;
                return false;
            }
        }
    }
}

// Shared-memory matrix descriptor of a K-major operand tile stored as rows of 64 bytes
// with the 64-byte swizzle (as written by TMA with CU_TENSOR_MAP_SWIZZLE_64B): 8-row
// groups are 512 bytes apart (stride byte offset); the leading byte offset is not used
// for swizzled K-major tiles.
__device__ __forceinline__ uint64_t desc_k_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);   // bits 0-13: start address >> 4
    d |= static_cast<uint64_t>(1u) << 16;                   // bits 16-29: leading byte offset >> 4
    d |= static_cast<uint64_t>(512u >> 4) << 32;            // bits 32-45: stride byte offset >> 4
    d |= static_cast<uint64_t>(1u) << 46;                   // bits 46-47: descriptor version 1
    d |= static_cast<uint64_t>(4u) << 61;                   // bits 61-63: 64-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4)                                  // D format: F32
           | (1u << 7)                                // A format: BF16
           | (1u << 10)                               // B format: BF16
           | (static_cast<uint32_t>(n >> 3) << 17)    // N / 8
           | (static_cast<uint32_t>(m >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ kernel

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_gemm3_tc(const __grid_constant__ CUtensorMap tm_dhi, const __grid_constant__ CUtensorMap tm_dlo,
               const __grid_constant__ CUtensorMap tm_xhi, const __grid_constant__ CUtensorMap tm_xlo,
               const Params p) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)p.stages * p.stage_bytes);
    uint64_t *empty = full + MAX_STAGES;
    uint64_t *acc_full = empty + MAX_STAGES;
    uint64_t *acc_empty = acc_full + 1;
    uint64_t *drain = acc_empty + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t G = gridDim.x;
    const int64_t u_begin = p.units * (int64_t)blockIdx.x / G;
    const int64_t u_end = p.units * ((int64_t)blockIdx.x + 1) / G;

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.stages; ++s) {
            mbar_init(smem_u32(full + s), 1);
            mbar_init(smem_u32(empty + s), 1);
        }
        mbar_init(smem_u32(acc_full), 1);
        mbar_init(smem_u32(acc_empty), 4);
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t smem_base = smem_u32(smem);

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- TMA producer
        int64_t it = 0;
        int64_t last_it[MAX_STAGES];
        for (int s = 0; s < MAX_STAGES; ++s) last_it[s] = -1;
        bool aborted = false;
        for (int64_t u = u_begin; u < u_end; ++u, ++it) {
            const int s = (int)(it % p.stages);
            const uint32_t ph = (uint32_t)((it / p.stages) & 1);
            if (!mbar_wait(smem_u32(empty + s), ph ^ 1u, p, 1, abort_flag)) {
                aborted = true;
                break;
            }
            const int tile = (int)(u / p.kblocks), kb = (int)(u % p.kblocks);
            const uint32_t base = smem_base + (uint32_t)s * p.stage_bytes;
            const uint32_t fb = smem_u32(full + s);
            mbar_expect_tx(fb, p.stage_bytes);
            tma_load_2d(base, &tm_dhi, fb, kb * BK, tile * BM);
            tma_load_2d(base + A_BYTES, &tm_dlo, fb, kb * BK, tile * BM);
            for (int j = 0; j < p.nsplit; ++j) {
                tma_load_2d(base + 2 * A_BYTES + (uint32_t)(j * p.nchunk * ROWB), &tm_xhi, fb, kb * BK, j * p.nchunk);
                tma_load_2d(base + 2 * A_BYTES + p.b_bytes + (uint32_t)(j * p.nchunk * ROWB), &tm_xlo, fb, kb * BK,
                            j * p.nchunk);
            }
            last_it[s] = it;
        }
        if (aborted) {
            // wait (bounded) for the copies already issued before leaving
            for (int s = 0; s < p.stages; ++s)
                if (last_it[s] >= 0) {
                    volatile int no_abort = 0;
                    mbar_wait(smem_u32(full + s), (uint32_t)((last_it[s] / p.stages) & 1), p, 1, &no_abort);
                }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------- MMA issuer
        const uint32_t idesc = idesc_bf16(BM, p.nchunk);
        int64_t it = 0, seg = 0;
        int64_t u = u_begin;
        bool aborted = false;
        while (u < u_end && !aborted) {
            const int64_t tile = u / p.kblocks;
            const int64_t seg_end = u_end < (tile + 1) * p.kblocks ? u_end : (tile + 1) * p.kblocks;
            if (!mbar_wait(smem_u32(acc_empty), (uint32_t)((seg & 1) ^ 1), p, 3, abort_flag)) break;
            tc_fence_after();
            bool first = true;
            for (; u < seg_end; ++u, ++it) {
                const int s = (int)(it % p.stages);
                const uint32_t ph = (uint32_t)((it / p.stages) & 1);
                if (!mbar_wait(smem_u32(full + s), ph, p, 2, abort_flag)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint32_t base = smem_base + (uint32_t)s * p.stage_bytes;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint32_t koff = (uint32_t)ks * 32u;   // 16 bf16 = 32 bytes along K
                    const uint64_t a_hi = desc_k_sw64(base + koff);
                    const uint64_t a_lo = desc_k_sw64(base + A_BYTES + koff);
                    for (int j = 0; j < p.nsplit; ++j) {
                        const uint32_t boff = (uint32_t)(j * p.nchunk * ROWB) + koff;
                        const uint64_t b_hi = desc_k_sw64(base + 2 * A_BYTES + boff);
                        const uint64_t b_lo = desc_k_sw64(base + 2 * A_BYTES + p.b_bytes + boff);
                        const uint32_t d = tmem + (uint32_t)(j * p.nchunk);
                        umma_bf16(d, a_hi, b_hi, idesc, first ? 0u : 1u);
                        umma_bf16(d, a_hi, b_lo, idesc, 1u);
                        umma_bf16(d, a_lo, b_hi, idesc, 1u);
                    }
                    first = false;
                }
                umma_commit(smem_u32(empty + s));
            }
            if (aborted) break;
            umma_commit(smem_u32(acc_full));
            ++seg;
        }
        // every MMA this thread issued has completed once `drain` flips
        umma_commit(smem_u32(drain));
        volatile int no_abort = 0;
        mbar_wait(smem_u32(drain), 0u, p, 5, &no_abort);
    } else if (warp >= 2) {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3;
        const int row_in_tile = quad * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const bool vec = ((p.ldu & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.U) & 15) == 0);
        int64_t seg = 0;
        int64_t u = u_begin;
        while (u < u_end) {
            const int64_t tile = u / p.kblocks;
            const int64_t seg_end = u_end < (tile + 1) * p.kblocks ? u_end : (tile + 1) * p.kblocks;
            const bool whole = (u == tile * p.kblocks) && (seg_end == (tile + 1) * p.kblocks);
            if (!mbar_wait(smem_u32(acc_full), (uint32_t)(seg & 1), p, 4, abort_flag)) break;
            tc_fence_after();
            const int64_t row = tile * BM + row_in_tile;
            float *dst_row = p.U + row * p.ldu;
            for (int c0 = 0; c0 < p.cpad; c0 += 32) {
                float v[32];
                tmem_ld32(lane_base + (uint32_t)c0, v);
                if (row >= p.n || c0 >= p.ncols) continue;
                float *dst = dst_row + c0;
                if (vec && c0 + 32 <= p.ncols) {
                    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float4 w = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                        if (whole)
                            d4[q] = w;
                        else
                            atomicAdd(d4 + q, w);
                    }
                } else {
                    for (int q = 0; q < 32 && c0 + q < p.ncols; ++q) {
                        if (whole)
                            dst[q] = v[q];
                        else
                            atomicAdd(dst + q, v[q]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(acc_empty));
            u = seg_end;
            ++seg;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
    }
}

// ------------------------------------------------------------------ host side

// 2-D bf16 tensor map: `rows` rows of `inner` elements (row pitch `pitch_elems`), box of
// BK x box_rows elements, 64-byte swizzle.
inline bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint64_t pitch_elems,
                     uint32_t box_rows, std::string *msg) {
    EncodeTiledFn fn = encode_fn(msg);
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {pitch_elems * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (msg) *msg = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        return false;
    }
    return true;
}

// CTAs of one launch: one per SM when there are at least as many row tiles as SMs
// (stream-K ranges of >= one tile: a tile is shared by at most two CTAs); otherwise each
// tile is split in at most two halves, which keeps the result deterministic.
inline int64_t grid_size(int64_t mtiles, int num_sms) {
    if (mtiles >= num_sms) return num_sms;
    int64_t split = num_sms / mtiles;
    if (split > 2) split = 2;
    if (split < 1) split = 1;
    return mtiles * split;
}

// Launch for one group of <= 512 accumulator columns.  Returns cudaSuccess or an error;
// *msg describes failures that are not CUDA runtime errors.
inline cudaError_t launch_group(const __nv_bfloat16 *Dhi, const __nv_bfloat16 *Dlo, int64_t n, int64_t npad,
                                const __nv_bfloat16 *Xhi, const __nv_bfloat16 *Xlo, int cpad, float *U, int64_t ldu,
                                int64_t ncols, int num_sms, int *err, cudaStream_t s, std::string *msg, int stages_req = 0) {
    Params p{};
    p.n = n;
    p.ldu = ldu;
    p.ncols = ncols;
    p.kblocks = (int)(npad / BK);
    const int64_t mtiles = npad / BM;
    p.units = mtiles * p.kblocks;
    p.cpad = cpad;
    p.nsplit = (cpad + 255) / 256;
    p.nchunk = cpad / p.nsplit;
    p.b_bytes = (uint32_t)cpad * ROWB;
    p.stage_bytes = 2 * A_BYTES + 2 * p.b_bytes;
    p.stages = (int)((kMaxDynSmem - 2048) / p.stage_bytes);
    if (p.stages > MAX_STAGES) p.stages = MAX_STAGES;
    if (stages_req >= 2 && stages_req < p.stages) p.stages = stages_req;   // a shallower pipeline (autotuner)
    int tc = 32;
    while (tc < cpad) tc <<= 1;
    p.tmem_cols = tc;
    p.U = U;
    p.err = err;
    p.timeout_ns = 2000000000ull;
    if (p.stages < 2 || p.nchunk % 16 != 0 || p.nchunk > 256) {
        if (msg) *msg = "gemm_tc: unsupported column count";
        return cudaErrorInvalidValue;
    }
    CUtensorMap m_dhi, m_dlo, m_xhi, m_xlo;
    if (!make_map(&m_dhi, Dhi, npad, npad, npad, BM, msg) || !make_map(&m_dlo, Dlo, npad, npad, npad, BM, msg) ||
        !make_map(&m_xhi, Xhi, npad, cpad, npad, p.nchunk, msg) ||
        !make_map(&m_xlo, Xlo, npad, cpad, npad, p.nchunk, msg))
        return cudaErrorInvalidValue;
    const int64_t grid = grid_size(mtiles, num_sms);
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + 256;
    static std::atomic<uint64_t> smem_set{0};
    if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
    cudaError_t e = allow_max_smem(k_gemm3_tc, smem_set);
    if (e != cudaSuccess) return e;
    k_gemm3_tc<<<(unsigned)grid, NUM_THREADS, smem, s>>>(m_dhi, m_dlo, m_xhi, m_xlo, p);
    return cudaGetLastError();
}

// Full launch: accumulator columns in groups of at most 512.  U must not alias X.
inline cudaError_t gemm3_tc(const __nv_bfloat16 *Dhi, const __nv_bfloat16 *Dlo, int64_t n, int64_t npad,
                            const __nv_bfloat16 *Xhi, const __nv_bfloat16 *Xlo, int64_t cpad, float *U, int64_t ldu,
                            int num_sms, int *err, cudaStream_t s, int *launches, std::string *msg, int stages_req = 0) {
    if (npad % BM != 0 || cpad % 32 != 0 || cpad < ldu || ldu < 1) {
        if (msg) *msg = "gemm_tc: bad shape";
        return cudaErrorInvalidValue;
    }
    // tiles shared by two CTAs are summed with atomics onto zeros
    if (grid_size(npad / BM, num_sms) != npad / BM) {
        cudaError_t e = cudaMemsetAsync(U, 0, sizeof(float) * (size_t)n * (size_t)ldu, s);
        if (e != cudaSuccess) return e;
    }
    for (int64_t c0 = 0; c0 < ldu; c0 += 512) {
        const int group = (int)((cpad - c0) < 512 ? (cpad - c0) : 512);
        const int64_t valid = (ldu - c0) < group ? (ldu - c0) : group;
        cudaError_t e = launch_group(Dhi, Dlo, n, npad, Xhi + c0 * npad, Xlo + c0 * npad, group, U + c0, ldu, valid,
                                     num_sms, err, s, msg, stages_req);
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

}  // namespace tc
}  // namespace wfq
