// Matrix-free tensor-core product U = D X for the mixed operator (sm_103a): the tiles of
// D (Eq. 3, widths from Eq. 4) are generated in shared memory from the atom records
// instead of being read from a stored matrix, then contracted with the three bf16
// products of gemm_tc.cuh.
//
// Roles (18 warps):
//   warp 0     : TMEM allocation; one lane loads, per stage, the Xhi / Xlo tiles (TMA) and
//                the 32 atom records of the stage's K block (bulk copy, own barrier).
//   warp 1     : one lane issues tcgen05.mma (three products per 16-atom K step).
//   warps 2-17 : generate the 128 x 32 D tile of every stage -- one row per thread, one
//                16-byte chunk (8 atoms) per group of four warps -- as bf16 hi and lo,
//                written straight into the 64-byte-swizzled K-major layout the MMA
//                descriptors expect; then a proxy fence and one arrival per warp on the
//                stage's full-barrier.
//   warps 2-5  : also the epilogue (TMEM -> registers -> U), as in gemm_tc.cuh.
// Work split and waits are those of gemm_tc.cuh (stream-K over (row tile, k block) units,
// at most two CTAs per tile, bounded barrier waits).
#pragma once

#include "gemm_tc.cuh"

namespace wfq {
namespace tc {

constexpr int MF_GEN_WARPS = 16;
constexpr uint32_t MF_ATOM_BYTES = BK * 16;   // 32 float4 atom records per stage
constexpr int MF_THREADS = 64 + 32 * MF_GEN_WARPS;

struct MfParams {
    Params p;
    const float4 *atoms;     // npad records (x, y, z, width); rows/columns >= n are zero in D
    const float4 *atoms_p;   // the same by atom pairs: (x0, x1, y0, y1), (z0, z1, w0, w1)
};

// D_ik of Eq. 3 in FP32.  Beyond r = 4 sigma, erfc < 1.6e-8 and erf(r/sigma) rounds to 1
// in FP32, so 1/r is returned without erf.
__device__ __forceinline__ float d_pair_f32(float4 a, float4 b, float wa2) {
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float s2 = wa2 + b.w * b.w;
    const float rinv = rsqrtf(r2);
    if (r2 >= 16.0f * s2) return rinv;
    return erff(r2 * rinv * rsqrtf(s2)) * rinv;
}

// 1/sqrt(x) in one MUFU operation (flush-to-zero approximate form, relative error below
// 2^-22; r^2 is never subnormal here and the result is kept to 16 bits in the hi/lo split).
__device__ __forceinline__ float rsqrt_mufu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// (a, b) -> bf16 pair (a in the low half), one conversion instruction for both
__device__ __forceinline__ uint32_t bf16x2_rn(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

__global__ void __launch_bounds__(MF_THREADS, 1)
    k_gemm3_mf(const __grid_constant__ CUtensorMap tm_xhi, const __grid_constant__ CUtensorMap tm_xlo,
               const MfParams mp) {
    const Params &p = mp.p;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)p.stages * p.stage_bytes);
    uint64_t *empty = full + MAX_STAGES;
    uint64_t *acc_full = empty + MAX_STAGES;
    uint64_t *acc_empty = acc_full + 1;
    uint64_t *drain = acc_empty + 1;
    uint64_t *atoms_full = drain + 1;   // MAX_STAGES barriers: k-atom records landed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(atoms_full + MAX_STAGES);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t atoms_off = 2 * A_BYTES + 2 * p.b_bytes;   // k-atom records inside a stage

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t G = gridDim.x;
    const int64_t u_begin = p.units * (int64_t)blockIdx.x / G;
    const int64_t u_end = p.units * ((int64_t)blockIdx.x + 1) / G;

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.stages; ++s) {
            mbar_init(smem_u32(full + s), 1 + MF_GEN_WARPS);
            mbar_init(smem_u32(empty + s), 1);
            mbar_init(smem_u32(atoms_full + s), 1);
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
    const uint32_t b_tx = 2u * p.b_bytes;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------------- TMA producer (X only)
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
                const int kb = (int)(u % p.kblocks);
                const uint32_t base = smem_base + (uint32_t)s * p.stage_bytes;
                const uint32_t fb = smem_u32(full + s);
                const uint32_t ab = smem_u32(atoms_full + s);
                mbar_expect_tx(ab, MF_ATOM_BYTES);
                bulk_load(base + atoms_off, mp.atoms_p + (int64_t)kb * BK, MF_ATOM_BYTES, ab);
                mbar_expect_tx(fb, b_tx);
                for (int j = 0; j < p.nsplit; ++j) {
                    tma_load_2d(base + 2 * A_BYTES + (uint32_t)(j * p.nchunk * ROWB), &tm_xhi, fb, kb * BK,
                                j * p.nchunk);
                    tma_load_2d(base + 2 * A_BYTES + p.b_bytes + (uint32_t)(j * p.nchunk * ROWB), &tm_xlo, fb,
                                kb * BK, j * p.nchunk);
                }
                last_it[s] = it;
            }
            if (aborted)
                for (int s = 0; s < p.stages; ++s)
                    if (last_it[s] >= 0) {
                        volatile int no_abort = 0;
                        const uint32_t par = (uint32_t)((last_it[s] / p.stages) & 1);
                        mbar_wait(smem_u32(atoms_full + s), par, p, 1, &no_abort);
                        mbar_wait(smem_u32(full + s), par, p, 1, &no_abort);
                    }
        }
    } else if (warp == 1) {
        if (lane == 0) {
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
                        const uint32_t koff = (uint32_t)ks * 32u;
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
            umma_commit(smem_u32(drain));
            volatile int no_abort = 0;
            mbar_wait(smem_u32(drain), 0u, p, 5, &no_abort);
        }
    } else {
        // ---------------------------------------------------------- D-tile generators
        const int gt = threadIdx.x - 64;           // 0..511
        const int row = gt & (BM - 1);             // tile row of this thread
        const int kc = gt >> 7;                    // 16-byte chunk (8 atoms) of the 64-byte row
        const bool epi = warp < 6;                 // warps 2-5 also run the epilogue
        const int quad = warp & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const int epi_row = quad * 32 + lane;
        const bool vec = ((p.ldu & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.U) & 15) == 0);
        const float eta_from_w = 0.7978845608028654f;   // sqrt(2/pi): eta = sqrt(2/pi) / width (Eq. 4)
        int64_t it = 0, seg = 0;
        int64_t u = u_begin;
        bool aborted = false;
        while (u < u_end && !aborted) {
            const int64_t tile = u / p.kblocks;
            const int64_t seg_end = u_end < (tile + 1) * p.kblocks ? u_end : (tile + 1) * p.kblocks;
            const int64_t seg_begin = u;
            const int gi = (int)(tile * BM + row);
            const float4 ai = mp.atoms[gi];
            const bool row_ok = gi < p.n;
            const float wa2 = ai.w * ai.w;
            const float eta_i = eta_from_w / ai.w;
            // the row atom as packed operands (the same value in both lanes)
            const float2 aix2 = make_float2(ai.x, ai.x), aiy2 = make_float2(ai.y, ai.y);
            const float2 aiz2 = make_float2(ai.z, ai.z), wa2_2 = make_float2(wa2, wa2);
            for (; u < seg_end; ++u, ++it) {
                const int s = (int)(it % p.stages);
                const uint32_t ph = (uint32_t)((it / p.stages) & 1);
                // the k-atom records land only after the stage was released by the MMAs,
                // so this one wait covers both
                if (!mbar_wait(smem_u32(atoms_full + s), ph, p, 6, abort_flag)) {
                    aborted = true;
                    break;
                }
                const int k0 = (int)(u % p.kblocks) * BK;
                const uint32_t base = smem_base + (uint32_t)s * p.stage_bytes;
                const float4 *atoms_s = reinterpret_cast<const float4 *>(smem + (size_t)s * p.stage_bytes + atoms_off);
                {
                    const int kb0 = k0 + kc * 8;
                    float dv[8], r2v[8], s2v[8];
                    // the chunk's 8 atoms as 4 pairs, two k-atoms per packed FP32x2 operation
                    // (per lane the same operations, in the same order, as for one atom)
                    float nmin = 1.f;   // min of r^2 - 16 s^2 over the chunk: < 0 for a near pair
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 xy = atoms_s[kc * 8 + 2 * q], zw = atoms_s[kc * 8 + 2 * q + 1];
                        const float2 dx = __fadd2_rn(aix2, make_float2(-xy.x, -xy.y));
                        const float2 dy = __fadd2_rn(aiy2, make_float2(-xy.z, -xy.w));
                        const float2 dz = __fadd2_rn(aiz2, make_float2(-zw.x, -zw.y));
                        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                        const float2 bw = make_float2(zw.z, zw.w);
                        const float2 s2 = __ffma2_rn(bw, bw, wa2_2);
                        r2v[2 * q] = r2.x;
                        r2v[2 * q + 1] = r2.y;
                        s2v[2 * q] = s2.x;
                        s2v[2 * q + 1] = s2.y;
                        // far pairs: 1/r from one rsqrt (erf(r/sigma) rounds to 1 in FP32)
                        dv[2 * q] = rsqrt_mufu(r2.x);
                        dv[2 * q + 1] = rsqrt_mufu(r2.y);
                        // r^2 - 16 s^2 in one rounding: its sign is that of r^2 - 16 s^2 itself
                        const float2 t = __ffma2_rn(s2, make_float2(-16.f, -16.f), r2);
                        nmin = fminf(nmin, fminf(t.x, t.y));
                    }
                    const bool near = nmin < 0.f;
                    // near pairs (rare: only tiles close to the diagonal) take the erf branch,
                    // entered by a warp only when one of its lanes needs it
                    if (__any_sync(0xffffffffu, near)) {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (r2v[e] < 16.0f * s2v[e]) dv[e] = erff(r2v[e] * dv[e] * rsqrtf(s2v[e])) * dv[e];
                    }
                    if (gi >= kb0 && gi < kb0 + 8) {                      // D_ii = eta_i
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (gi == kb0 + e) dv[e] = eta_i;
                    }
                    if (!row_ok || kb0 + 8 > p.n) {                       // padding rows / columns
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (!row_ok || kb0 + e >= p.n) dv[e] = 0.f;
                    }
                    // hi = bf16(D), lo = bf16(D - hi), two entries per conversion
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const uint32_t h = bf16x2_rn(dv[e], dv[e + 1]);
                        const float2 h01 = make_float2(__uint_as_float(h << 16), __uint_as_float(h & 0xffff0000u));
                        const float2 d = __fadd2_rn(make_float2(dv[e], dv[e + 1]), make_float2(-h01.x, -h01.y));
                        hw[e >> 1] = h;
                        lw[e >> 1] = bf16x2_rn(d.x, d.y);
                    }
                    // 64-byte swizzle: 16-byte chunk index XOR (row / 2) mod 4
                    const uint32_t off = (uint32_t)row * 64u + (uint32_t)((kc ^ ((row >> 1) & 3)) * 16);
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + off), "r"(hw[0]), "r"(hw[1]),
                                 "r"(hw[2]), "r"(hw[3])
                                 : "memory");
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + A_BYTES + off), "r"(lw[0]),
                                 "r"(lw[1]), "r"(lw[2]), "r"(lw[3])
                                 : "memory");
                }
                // generic-proxy writes -> visible to the tensor cores' async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(full + s));
            }
            if (aborted || !epi) {
                ++seg;
                continue;
            }
            // ---------------------------------------------------------- epilogue (warps 2-5)
            const bool whole_tile = (seg_begin == tile * p.kblocks) && (seg_end == (tile + 1) * p.kblocks);
            if (!mbar_wait(smem_u32(acc_full), (uint32_t)(seg & 1), p, 4, abort_flag)) break;
            tc_fence_after();
            const int64_t orow = tile * BM + epi_row;
            float *dst_row = p.U + orow * p.ldu;
            for (int c0 = 0; c0 < p.cpad; c0 += 32) {
                float v[32];
                tmem_ld32(lane_base + (uint32_t)c0, v);
                if (orow >= p.n || c0 >= p.ncols) continue;
                float *dst = dst_row + c0;
                if (vec && c0 + 32 <= p.ncols) {
                    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        float4 w = make_float4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
                        if (whole_tile)
                            d4[qq] = w;
                        else
                            atomicAdd(d4 + qq, w);
                    }
                } else {
                    for (int qq = 0; qq < 32 && c0 + qq < p.ncols; ++qq) {
                        if (whole_tile)
                            dst[qq] = v[qq];
                        else
                            atomicAdd(dst + qq, v[qq]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(acc_empty));
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

// One launch for a group of <= 512 accumulator columns.
inline cudaError_t launch_group_mf(const float4 *atoms, const float4 *atoms_p, int64_t n, int64_t npad,
                                   const __nv_bfloat16 *Xhi,
                                   const __nv_bfloat16 *Xlo, int cpad, float *U, int64_t ldu, int64_t ncols,
                                   int num_sms, int *err, cudaStream_t s, std::string *msg,
                                   int stages_req = 0) {
    MfParams mp{};
    Params &p = mp.p;
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
    p.stage_bytes = (2 * A_BYTES + 2 * p.b_bytes + MF_ATOM_BYTES + 1023) / 1024 * 1024;
    p.stages = (int)((kMaxDynSmem - 2048) / p.stage_bytes);
    if (p.stages > MAX_STAGES) p.stages = MAX_STAGES;
    if (stages_req >= 2 && stages_req < p.stages) p.stages = stages_req;   // a shallower pipeline (autotuner)
    int tcols = 32;
    while (tcols < cpad) tcols <<= 1;
    p.tmem_cols = tcols;
    p.U = U;
    p.err = err;
    p.timeout_ns = 4000000000ull;
    mp.atoms = atoms;
    mp.atoms_p = atoms_p;
    if (p.stages < 2 || p.nchunk % 16 != 0 || p.nchunk > 256) {
        if (msg) *msg = "gemm_mf: unsupported column count";
        return cudaErrorInvalidValue;
    }
    CUtensorMap m_xhi, m_xlo;
    if (!make_map(&m_xhi, Xhi, npad, cpad, npad, p.nchunk, msg) || !make_map(&m_xlo, Xlo, npad, cpad, npad, p.nchunk, msg))
        return cudaErrorInvalidValue;
    const int64_t grid = grid_size(mtiles, num_sms);
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + 512;
    static std::atomic<uint64_t> smem_set{0};
    if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
    cudaError_t e = allow_max_smem(k_gemm3_mf, smem_set);
    if (e != cudaSuccess) return e;
    k_gemm3_mf<<<(unsigned)grid, MF_THREADS, smem, s>>>(m_xhi, m_xlo, mp);
    return cudaGetLastError();
}

inline cudaError_t gemm3_mf(const float4 *atoms, const float4 *atoms_p, int64_t n, int64_t npad,
                            const __nv_bfloat16 *Xhi,
                            const __nv_bfloat16 *Xlo, int64_t cpad, float *U, int64_t ldu, int num_sms, int *err,
                            cudaStream_t s, int *launches, std::string *msg, int stages_req = 0) {
    if (npad % BM != 0 || cpad % 32 != 0 || cpad < ldu || ldu < 1) {
        if (msg) *msg = "gemm_mf: bad shape";
        return cudaErrorInvalidValue;
    }
    if (grid_size(npad / BM, num_sms) != npad / BM) {
        cudaError_t e = cudaMemsetAsync(U, 0, sizeof(float) * (size_t)n * (size_t)ldu, s);
        if (e != cudaSuccess) return e;
    }
    for (int64_t c0 = 0; c0 < ldu; c0 += 512) {
        const int group = (int)((cpad - c0) < 512 ? (cpad - c0) : 512);
        const int64_t valid = (ldu - c0) < group ? (ldu - c0) : group;
        cudaError_t e = launch_group_mf(atoms, atoms_p, n, npad, Xhi + c0 * npad, Xlo + c0 * npad, group, U + c0, ldu, valid,
                                        num_sms, err, s, msg, stages_req);
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

}  // namespace tc
}  // namespace wfq
