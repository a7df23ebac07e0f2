// BF16 GEMM of the learned level's dense layers on the 5th-generation tensor
// cores (sm_103a): C[M x N] = A[M x K] . B[N x K]^T, both operands K-major BF16
// in global memory, FP32 accumulation in tensor memory (TMEM).
//
// One CTA computes a 128-row tile of C across all N <= 256 columns:
//   * one thread streams 128 x 64 tiles of A and N x 64 tiles of B into a
//     ring of shared-memory stages with TMA (cp.async.bulk.tensor, 128-byte
//     swizzle, rows beyond M or K read as zeros), each stage guarded by a
//     "full" mbarrier (transaction count) and an "empty" one;
//   * one thread issues tcgen05.mma (kind::f16, M = 128, N, K = 16 per
//     instruction, four per stage) into a 128-lane x N-column FP32 accumulator
//     in TMEM and frees each stage with tcgen05.commit;
//   * all four warps then read their 32 TMEM lanes (= rows) with tcgen05.ld and
//     apply the epilogue: + bias[n], ReLU, * (mask[m][n] > 0), FP32 and/or BF16
//     output, each thread 32 consecutive columns of its row per tcgen05.ld
//     with 16-byte loads and stores.
// Every mbarrier wait is bounded: after kMbarPolls polls it records
// kErrTimeout in the error word and the CTA skips to the epilogue, which still
// frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "dk_kernels.h"

namespace dk {

namespace {

constexpr int kTM = 128;                        // rows of a CTA tile (TMEM lanes)
constexpr int kTK = 64;                         // K of a stage: 64 BF16 = one 128-byte swizzle row
constexpr int kStages = 2;   // two stages: 99 KB at N = 256, so two CTAs share an SM
constexpr unsigned kMbarPolls = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait for the phase with parity `parity` of the mbarrier to complete; false
// after kMbarPolls polls (the timeout is recorded) or once `skip` is set.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned* err) {
    const uint32_t addr = smem_u32(bar);
    for (unsigned i = 0; i < kMbarPolls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    atomicOr(err, kErrTimeout);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzling: rows of 128 bytes, groups of 8 rows 1024 bytes
// apart (stride byte offset), descriptor version 1, swizzle mode 128 B.
__device__ __forceinline__ uint64_t umma_desc(const void* tile) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((smem_u32(tile) >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(1) << 16;              // leading byte offset (unused with 128 B swizzle, K-major)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;      // stride byte offset: 8 rows x 128 B
    d |= static_cast<uint64_t>(1) << 46;              // descriptor version
    d |= static_cast<uint64_t>(2) << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
           (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN>
constexpr size_t umma_smem_bytes() {
    return 1024 /* alignment slack */ + (size_t)kStages * (kTM + BN) * kTK * sizeof(__nv_bfloat16) +
           (2 * kStages + 1) * sizeof(uint64_t) + 16;
}

template <int BN>
__global__ void __launch_bounds__(128, 1)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, const GemmArgs g,
                     unsigned* err) {
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256 && (BN & (BN - 1)) == 0, "N tile: power of two in [32, 256]");
    extern __shared__ unsigned char umma_shared[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(umma_shared) + 1023) & ~static_cast<uintptr_t>(1023));
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(base);                 // [stages][128][64]
    __nv_bfloat16* sB = sA + (size_t)kStages * kTM * kTK;                        // [stages][BN][64]
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + (size_t)kStages * BN * kTK);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kTM;
    const int ktiles = (g.K + kTK - 1) / kTK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of the K tiles into the stage ring
        constexpr uint32_t bytes = (kTM + BN) * kTK * sizeof(__nv_bfloat16);
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % kStages;
            if (kt >= kStages && !mbar_wait(&empty[s], ((kt / kStages) - 1) & 1, err)) break;
            mbar_expect_tx(&full[s], bytes);
            tma_load_2d(sA + (size_t)s * kTM * kTK, &tA, kt * kTK, m0, &full[s]);
            tma_load_2d(sB + (size_t)s * BN * kTK, &tB, kt * kTK, 0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: four K = 16 steps per stage (32 bytes along the swizzled rows)
        constexpr uint32_t idesc = umma_idesc(kTM, BN);
        bool ok = true;
        for (int kt = 0; kt < ktiles && ok; ++kt) {
            const int s = kt % kStages;
            ok = mbar_wait(&full[s], (kt / kStages) & 1, err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = umma_desc(sA + (size_t)s * kTM * kTK);
            const uint64_t db = umma_desc(sB + (size_t)s * BN * kTK);
#pragma unroll
            for (int kk = 0; kk < kTK / 16; ++kk)
                umma_bf16(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (kt | kk) != 0 ? 1u : 0u);
            umma_commit(&empty[s]);
        }
        umma_commit(done);
    }
    // epilogue: warp w reads TMEM lanes 32w .. 32w + 31 (rows of the tile)
    const bool ready = mbar_wait(done, 0, err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = m0 + warp * 32 + lane;
    if (ready) {
#pragma unroll 1
        for (int c0 = 0; c0 < BN && c0 < g.N; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c0), v);
            if (m >= g.M) continue;
            // this thread's 32 consecutive columns of row m: 16-byte loads and
            // stores where the whole chunk is inside N and the row is aligned
            const bool full = c0 + 32 <= g.N;
            float x[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = __uint_as_float(v[j]);
            if (g.bias) {
                if (full && (reinterpret_cast<uintptr_t>(g.bias + c0) & 15) == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 b = *reinterpret_cast<const float4*>(g.bias + c0 + j);
                        x[j] += b.x; x[j + 1] += b.y; x[j + 2] += b.z; x[j + 3] += b.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < g.N) x[j] += g.bias[c0 + j];
                }
            }
            if (g.relu)
#pragma unroll
                for (int j = 0; j < 32; ++j) x[j] = fmaxf(x[j], 0.f);
            if (g.mask) {
                const __nv_bfloat16* mr = g.mask + (long long)m * g.ldm + c0;
                if (full && (reinterpret_cast<uintptr_t>(mr) & 15) == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j += 8) {
                        const uint4 w = *reinterpret_cast<const uint4*>(mr + j);
                        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&w);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (!(__bfloat162float(h[i]) > 0.f)) x[j + i] = 0.f;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < g.N && !(__bfloat162float(mr[j]) > 0.f)) x[j] = 0.f;
                }
            }
            if (g.C) {
                float* cr = g.C + (long long)m * g.ldc + c0;
                if (full && (reinterpret_cast<uintptr_t>(cr) & 15) == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *reinterpret_cast<float4*>(cr + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < g.N) cr[j] = x[j];
                }
            }
            if (g.Cb) {
                __nv_bfloat16* br = g.Cb + (long long)m * g.ldcb + c0;
                if (full && (reinterpret_cast<uintptr_t>(br) & 15) == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j += 8) {
                        uint4 w;
                        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
                        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(x[j + 2 * i], x[j + 2 * i + 1]);
                        *reinterpret_cast<uint4*>(br + j) = w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < g.N) br[j] = __float2bfloat16_rn(x[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// BF16 transpose: out[c][r] = in[r][c] for an R x C row-major matrix, output
// rows ldo >= R elements apart.
__global__ void transpose_bf16_kernel(const __nv_bfloat16* in, int R, int C, __nv_bfloat16* out, int ldo) {
    __shared__ __nv_bfloat16 t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = by + i, c = bx + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = in[(size_t)r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = bx + i, r = by + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * ldo + r] = t[threadIdx.x][i];
    }
}

// ---------------------------------------------------------------- host side
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// Tensor map of a K-major BF16 matrix [rows][K] (row stride ld elements): box
// 64 (K) x box_rows, 128-byte swizzle, out-of-range elements read as zero.
bool encode_kmajor(CUtensorMap* map, const __nv_bfloat16* ptr, long long rows, long long K, long long ld,
                   int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t umma_launch(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, unsigned* err,
                        cudaStream_t st) {
    const cudaError_t attr = cudaFuncSetAttribute(umma_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)umma_smem_bytes<BN>());
    if (attr != cudaSuccess) return attr;
    const int tiles = (g.M + kTM - 1) / kTM;
    umma_gemm_kernel<BN><<<tiles, 128, umma_smem_bytes<BN>(), st>>>(ta, tb, g, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_tc(const GemmArgs& g, unsigned* err, cudaStream_t st) {
    // A [M][K] K-major (sak == 1, row stride sam), B given as [N][K] K-major
    // (sbk == 1, row stride sbn): C = A B^T
    if (g.sak != 1 || g.sbk != 1 || g.N < 1 || g.N > 256 || g.M < 1 || g.K < 1 || !err) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(g.A) & 15) || (reinterpret_cast<uintptr_t>(g.B) & 15) || (g.sam * 2) % 16 ||
        (g.sbn * 2) % 16)
        return cudaErrorInvalidValue;
    const int bn = g.N <= 32 ? 32 : g.N <= 64 ? 64 : g.N <= 128 ? 128 : 256;
    CUtensorMap ta, tb;
    if (!encode_kmajor(&ta, g.A, g.M, g.K, g.sam, kTM) || !encode_kmajor(&tb, g.B, g.N, g.K, g.sbn, bn))
        return cudaErrorInvalidValue;
    switch (bn) {
        case 32: return umma_launch<32>(ta, tb, g, err, st);
        case 64: return umma_launch<64>(ta, tb, g, err, st);
        case 128: return umma_launch<128>(ta, tb, g, err, st);
        default: return umma_launch<256>(ta, tb, g, err, st);
    }
}

cudaError_t launch_transpose_bf16(const __nv_bfloat16* in, int R, int C, __nv_bfloat16* out, int ldo,
                                  cudaStream_t st) {
    if (ldo < R) return cudaErrorInvalidValue;
    const dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    transpose_bf16_kernel<<<grid, block, 0, st>>>(in, R, C, out, ldo);
    return cudaGetLastError();
}

}  // namespace dk
