// BF16 tensor-core GEMM for the actor/critic MLPs on sm_103a: tcgen05.mma with the FP32
// accumulator in tensor memory, operands staged by TMA into 128-byte-swizzled shared memory,
// and the layer epilogues (bias + ELU, ELU derivative + bias-gradient column sums, split-K
// FP32 partials) fused into the TMEM read-back.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]     A: [M][K] bf16, B: [N][K] bf16, both K contiguous
//
// Every MLP product is cast into this K-major form by keeping transposed copies where needed:
//   forward  H_l = ELU(H_{l-1} W_l^T + b_l):    A = H_{l-1} [rows][in],  B = W_l [out][in]
//   input    dY_{l-1} = (dY_l W_l) * ELU'(H):   A = dY_l [rows][out],    B = W_l^T [in][out]
//   weight   dW_l = dY_l^T H_{l-1}:             A = dY_l^T [out][rows],  B = H_{l-1}^T [in][rows]
// The forward and input-gradient epilogues write their bf16 result both row-major and
// transposed, so the weight-gradient GEMM finds its operands K-major.
//
// CTA: 128 threads, one 128 x BN output tile, K in steps of 64 (one 128-byte swizzle row).
// warp 0 lane 0 issues TMA loads into a STAGES-deep ring (full/empty mbarriers); warp 1
// lane 0 issues 4 tcgen05.mma (K = 16 each) per stage and releases the stage with
// tcgen05.commit; after the last stage a commit signals the accumulator, and all four warps
// read their 32 TMEM lanes (= tile rows) back with tcgen05.ld.  Every mbarrier wait is bounded
// by the global timer; a wait that runs out records RL_ERR_TIMEOUT in the status word and the
// CTA skips the rest of its work, frees its tensor memory and returns.
#include <cuda.h>

#include "common.cuh"
#include "gemm_tc.cuh"

namespace rl {

namespace {

constexpr int TC_THREADS = 128;
constexpr int BM = 128, BK = 64;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false (and records the timeout) after WAIT_NS.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 256; ++i)
            if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > WAIT_NS) {
            set_status(status, RL_ERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor, K-major operand with 128-byte swizzle: 8-row x 128-byte
// atoms stacked every 1024 bytes (stride byte offset), leading byte offset unused, descriptor
// version 1 (bits 46-48), layout code 2 = SWIZZLE_128B (bits 61-63).  The tile base is 1024-byte
// aligned; the k-th 16-element slice inside the swizzle row starts 32 bytes further.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
template <int N>
__device__ __forceinline__ uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int BN>
struct TileCfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = BN >= 256 ? 3 : 4;
    static constexpr int SMEM = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/ + 4 * BN * 4 /*colsum per warp*/;
};

template <int BN, int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
    using C = TileCfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::STAGES + 1);
    float* colsum_s = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE + 256);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + C::STAGES), tfull = smem_u32(bars + 2 * C::STAGES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.z / p.splits, sp = blockIdx.z % p.splits;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb0 = sp * p.kb_per_split;
    const int kb1 = min(p.kblocks, kb0 + p.kb_per_split);
    const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(tfull, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (EPI == EPI_ELU_GRAD)
        for (int i = threadIdx.x; i < 4 * BN; i += TC_THREADS) colsum_s[i] = 0.f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0 && nkb > 0) {
        // TMA producer
        const CUtensorMap* ma = &p.tmA[b];
        const CUtensorMap* mb = &p.tmB[b];
        for (int i = 0; i < nkb; ++i) {
            const int s = i % C::STAGES;
            const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.status)) break;
            const uint32_t sa = smem_u32(smem + s * C::STAGE);
            mbar_expect_tx(full0 + 8 * s, (uint32_t)C::STAGE);
            tma_load_2d(sa, ma, full0 + 8 * s, (kb0 + i) * BK, m0);
            tma_load_2d(sa + C::A_BYTES, mb, full0 + 8 * s, (kb0 + i) * BK, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_bf16<BN>();
        for (int i = 0; i < nkb; ++i) {
            const int s = i % C::STAGES;
            const uint32_t ph = (uint32_t)(i / C::STAGES) & 1u;
            if (!mbar_wait(full0 + 8 * s, ph, p.status)) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * C::STAGE);
            const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + C::A_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(tfull);   // arrives once every issued MMA has completed (immediately if none)
    }
    __syncwarp();

    // Epilogue: warp w owns TMEM lanes / tile rows 32w .. 32w + 31.
    const bool have = mbar_wait(tfull, 0u, p.status);
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    const bool row_ok = row < p.M;
    if (have) {
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (nkb == 0) {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.f;
            }
            const int col = n0 + c;
            if (EPI == EPI_STORE) {
                if (row_ok) {
                    float* dst = reinterpret_cast<float*>(p.C[b]) + (size_t)sp * p.split_stride + (size_t)row * p.ldc + col;
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
            } else {
                if (EPI == EPI_BIAS_ELU) {
                    const float* bias = p.bias[b] + col;
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = elu(v[j] + __ldg(bias + j));
                } else {   // EPI_ELU_GRAD
                    if (row_ok) {
                        const uint4* hp = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(p.H[b]) +
                                                                         (size_t)row * p.ldh + col);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint4 hv = __ldg(hp + q);
                            const __nv_bfloat16* h8 = reinterpret_cast<const __nv_bfloat16*>(&hv);
#pragma unroll
                            for (int j = 0; j < 8; ++j) v[8 * q + j] *= elu_grad_y(bf2f(h8[j]));
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = 0.f;
                    }
                }
                __align__(16) __nv_bfloat16 o[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) o[j] = f2bf(v[j]);
                if (row_ok) {
                    uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(p.C[b]) + (size_t)row * p.ldc + col);
#pragma unroll
                    for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
                    if (p.Ct[b]) {
                        __nv_bfloat16* ct = reinterpret_cast<__nv_bfloat16*>(p.Ct[b]) + (size_t)col * p.ldct + row;
#pragma unroll
                        for (int j = 0; j < 32; ++j) ct[(size_t)j * p.ldct] = o[j];
                    }
                }
                if (EPI == EPI_ELU_GRAD && p.colsum[b]) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float s = v[j];
#pragma unroll
                        for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o2);
                        if (lane == j) colsum_s[warp * BN + c + j] = s;   // per-warp slot, summed in order below
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (EPI == EPI_ELU_GRAD && p.colsum[b] && have)
        for (int i = threadIdx.x; i < BN; i += TC_THREADS)
            p.colsum[b][(size_t)blockIdx.x * p.N + n0 + i] =
                ((colsum_s[i] + colsum_s[BN + i]) + colsum_s[2 * BN + i]) + colsum_s[3 * BN + i];
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
    }
}

template <int BN, int EPI>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(tc_gemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, TileCfg<BN>::SMEM);
}

template <int BN, int EPI>
cudaError_t launch_cfg(const TcParams& p, cudaStream_t s) {
    using C = TileCfg<BN>;
    dim3 grid((p.M + BM - 1) / BM, p.N / BN, p.batch * p.splits);
    tc_gemm_kernel<BN, EPI><<<grid, TC_THREADS, C::SMEM, s>>>(p);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_bn(const TcParams& p, cudaStream_t s) {
    switch (p.bn) {
        case 64: return launch_cfg<64, EPI>(p, s);
        case 128: return launch_cfg<128, EPI>(p, s);
        case 256: return launch_cfg<256, EPI>(p, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_tc_gemm(const TcParams& p, cudaStream_t s) {
    if (p.M <= 0) return cudaSuccess;
    if (p.N % p.bn || p.kblocks <= 0 || p.splits <= 0 || p.batch < 1 || p.batch > 2) return cudaErrorInvalidValue;
    switch (p.epi) {
        case EPI_STORE: return launch_bn<EPI_STORE>(p, s);
        case EPI_BIAS_ELU: return launch_bn<EPI_BIAS_ELU>(p, s);
        case EPI_ELU_GRAD: return launch_bn<EPI_ELU_GRAD>(p, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- tensor maps (host)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

// 2D bf16 tensor [rows][cols] (cols contiguous, row stride ld elements), box 64 x box_rows,
// 128-byte swizzle, zero fill outside.  cols and ld must make 16-byte strides.
bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows) {
    EncodeTiledFn enc = get_encode();
    if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15u) || (ld * 2) % 16 || cols > ld) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Sets the dynamic shared-memory limit of every instantiation; called once per device before
// the first launch (and so before any stream capture).
cudaError_t tc_prepare() {
    cudaError_t e = cudaSuccess;
    e = e != cudaSuccess ? e : set_attr<64, EPI_STORE>();
    e = e != cudaSuccess ? e : set_attr<128, EPI_STORE>();
    e = e != cudaSuccess ? e : set_attr<256, EPI_STORE>();
    e = e != cudaSuccess ? e : set_attr<64, EPI_BIAS_ELU>();
    e = e != cudaSuccess ? e : set_attr<128, EPI_BIAS_ELU>();
    e = e != cudaSuccess ? e : set_attr<256, EPI_BIAS_ELU>();
    e = e != cudaSuccess ? e : set_attr<64, EPI_ELU_GRAD>();
    e = e != cudaSuccess ? e : set_attr<128, EPI_ELU_GRAD>();
    e = e != cudaSuccess ? e : set_attr<256, EPI_ELU_GRAD>();
    return e;
}

int tc_smem_bytes(int bn) {
    switch (bn) {
        case 64: return TileCfg<64>::SMEM;
        case 128: return TileCfg<128>::SMEM;
        case 256: return TileCfg<256>::SMEM;
    }
    return 0;
}

}  // namespace rl
