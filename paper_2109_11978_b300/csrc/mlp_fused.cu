// Fused forward of the actor / critic MLPs' three hidden layers (Sec. 2.2: ELU layers, here the
// 512-256-128 networks of the rough-terrain task) on sm_103a: one CTA per (128-row tile,
// network) carries its rows through all three layers, so that no hidden activation makes a round
// trip through global memory between layers and the three launches of the layer-by-layer form
// become one.
//
//   H_0 = ELU(X W_0^T + b_0),  H_1 = ELU(H_0 W_1^T + b_1),  H_2 = ELU(H_1 W_2^T + b_2)
//
// Each layer runs on tcgen05.mma (M = 128, N = 128, K = 16; bf16 operands, fp32 accumulator in
// tensor memory).  The weights stream through a ring of 16 KB shared-memory stages (128 rows x 64
// K, 128-byte swizzle) filled by TMA from L2; the activations stay in shared memory in the same
// K-major swizzled layout, written there by the epilogue warps (bias + ELU + bf16), where they
// serve directly as the next layer's A operand:
//
//   R0 (64 KB): X (TMA), then H_1 (epilogue of layer 1)
//   R1 (64 KB): a ring of four 64-column blocks of H_0, then H_2
//   TMEM: two 128-column buffers for layer-0 chunks and layer-2 chunks, 256 columns for layer 1
//
// Layer 0 runs in 128-column chunks; while the epilogue turns chunk c into two K blocks of H_0,
// the MMA warp issues chunk c + 1 and then layer 1's products over the K blocks of chunk c - 1
// (both of its 128-column halves accumulate at once), so layer 1 consumes H_0 as it is produced
// and H_0 needs four resident K blocks, not eight.  Layer 2 starts when layer 1's epilogue has
// written H_1.  The last layer's rows (and with store_hidden every layer's) leave by TMA store
// from the same shared-memory blocks.
//
// Roles (576 threads): warp 0 lanes 0-3 the TMA producer (stage i on lane i mod 4; lane 0 also
// the X tile), warp 1 lane 0 the MMA issuer and warp 1 the TMEM owner, warps 2-17 the epilogue
// (warp w reads TMEM lanes 32 (w mod 4) .. + 32, i.e. those rows, and a 32-column quarter of each
// 128-column chunk).  Every mbarrier wait is bounded (2 s on the global timer) and records
// RL_ERR_TIMEOUT; after a timeout every role stops issuing work, the epilogue warps still pass
// their named barriers (so none waits on a warp that gave up), copies and MMAs in flight are
// waited for (bounded) and the tensor memory is freed before the CTA returns.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "mlp_fused.cuh"
#include "tc_prims.cuh"

namespace rl {

namespace {

constexpr int MF_EPI_WARPS = 16;
constexpr int MF_THREADS = 64 + 32 * MF_EPI_WARPS;
constexpr int MF_KB = 16384;                      // one 64-column K block of 128 rows (bf16)
constexpr int MF_R0 = 4 * MF_KB;                  // X (K0 <= 256), then H_1 (N1 <= 256)
constexpr int MF_R1 = 4 * MF_KB;                  // H_0 ring, then H_2 (N2 <= 256)
constexpr int MF_BIAS = 4096;                     // b_0, b_1, b_2 (<= 1024 floats)
constexpr int MF_BAR = 1024;
constexpr int MF_FIXED = 1024 /*align*/ + MF_R0 + MF_R1 + MF_BIAS + MF_BAR;
constexpr int MF_STAGES = (227 * 1024 - MF_FIXED) / MF_KB;   // weight ring stages (5)
constexpr int MF_SMEM = MF_FIXED + MF_STAGES * MF_KB;
constexpr int MF_PROD = 4;                        // producer lanes
static_assert(MF_STAGES >= 2, "weight ring");
// barrier block: full[S], empty[S], xfull, accf[2], acce[2], h0r[2], l1f, h1r, drain, then the TMEM
// address and the abort flag
static_assert((2 * MF_STAGES + 11) * 8 + 8 <= MF_BAR, "barrier block");

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}

// the 512 epilogue threads (named barrier 1)
__device__ __forceinline__ void epi_sync() { asm volatile("barrier.sync 1, 512;" ::: "memory"); }

// Widths of one launch in blocks: layer 0's K blocks and 128-column chunks, layer 1's 128-column
// halves (K blocks = 2 x layer 0's chunks), layer 2's K blocks and chunks.
struct MfDims {
    int kb0, c0, h1, kb2, c2;
};

// The order in which weight blocks are consumed (and so loaded): layer 0's chunk c, then layer 1's
// products over H_0's K blocks 2 (c - 1), 2 (c - 1) + 1 (each for every 128-column half of H_1),
// ..., the last chunk's layer-1 blocks, then layer 2 chunk by chunk.  The producer and the MMA
// issuer both walk it, so the ring's stage order is the issue order by construction.
//   f.chunk(j)      a TMEM chunk j starts (layer 0: j = c; layer 2: j = c0 + c2; buffer j mod 2)
//   f.stage(l, row0, kb, akb, tcol, acc)   one weight block: W_l rows row0 .. + 128, K block kb,
//                   against A K block akb of the layer's input, into TMEM column tcol
//   f.chunk_done(j) the chunk's last block was issued
//   f.h0(cc)        H_0's K blocks of layer-0 chunk cc are needed next
//   f.l1_done()     layer 1's last block was issued
//   f.h1()          H_1 is needed next
template <class F>
__device__ __forceinline__ bool mf_walk(const MfDims& d, F& f) {
    for (int c = 0; c <= d.c0; ++c) {
        if (c < d.c0) {
            if (!f.chunk(c)) return false;
            for (int kb = 0; kb < d.kb0; ++kb)
                if (!f.stage(0, 128 * c, kb, kb, (uint32_t)(c & 1) * 128u, kb > 0)) return false;
            f.chunk_done(c);
        }
        if (c >= 1) {
            const int cc = c - 1;
            if (!f.h0(cc)) return false;
            for (int kb = 2 * cc; kb < 2 * cc + 2; ++kb)
                for (int h = 0; h < d.h1; ++h)
                    if (!f.stage(1, 128 * h, kb, kb & 3, 256u + 128u * (uint32_t)h, kb > 0)) return false;
        }
    }
    f.l1_done();
    if (!f.h1()) return false;
    for (int c2 = 0; c2 < d.c2; ++c2) {
        const int j = d.c0 + c2;
        if (!f.chunk(j)) return false;
        for (int kb = 0; kb < d.kb2; ++kb)
            if (!f.stage(2, 128 * c2, kb, kb, (uint32_t)(j & 1) * 128u, kb > 0)) return false;
        f.chunk_done(j);
    }
    return true;
}

// Number of weight blocks of a launch (the walk's stage count).
__device__ __forceinline__ int mf_stages_total(const MfDims& d) { return d.c0 * d.kb0 + 2 * d.c0 * d.h1 + d.c2 * d.kb2; }

// The TMA producer's side of the walk: stage k goes to ring slot k mod S from lane k mod 4, once
// the MMA has released the slot's previous block; stages outside [lo, hi) are skipped (the early
// fetch before the wait for the preceding kernel issues [0, S)).
struct MfProducer {
    const MlpParams* p;
    int net, lane, k, lo, hi, stop;
    uint32_t ring, full0, empty0;
    volatile int* abort;
    __device__ bool chunk(int) { return true; }
    __device__ void chunk_done(int) {}
    __device__ bool h0(int) { return true; }
    __device__ void l1_done() {}
    __device__ bool h1() { return true; }
    __device__ bool stage(int l, int row0, int kb, int, uint32_t, bool) {
        const int i = k++;
        if (i < lo || i >= hi || (i % MF_PROD) != lane) return true;
        const int s = i % MF_STAGES, u = i / MF_STAGES;
        if (u > 0 && !mbar_wait(empty0 + 8 * s, (uint32_t)(u - 1) & 1u, p->status, abort)) {
            *abort = 1;
            stop = i;
            return false;
        }
        mbar_expect_tx(full0 + 8 * s, (uint32_t)MF_KB);
        tma_load_2d(ring + (uint32_t)s * MF_KB, &p->tmW[net][l], full0 + 8 * s, 64 * kb, row0);
        return true;
    }
};

// The MMA issuer's side: four K = 16 products per weight block, the block's slot released by
// tcgen05.commit when they have read it; chunk and layer completions signalled the same way.
struct MfMma {
    uint32_t tmem, ring, r0, r1, idesc;
    uint32_t full0, empty0, accf, acce, h0r, l1f, h1r;
    int k;
    int* status;
    volatile int* abort;
    __device__ bool wait(uint32_t bar, uint32_t par) {
        if (!mbar_wait(bar, par, status, abort)) {
            *abort = 1;
            return false;
        }
        tc_fence_after();
        return true;
    }
    // buffer j mod 2's previous chunk (j - 2) has left TMEM
    __device__ bool chunk(int j) { return j < 2 || wait(acce + 8 * (j & 1), (uint32_t)((j >> 1) - 1) & 1u); }
    __device__ void chunk_done(int j) { mma_commit(accf + 8 * (j & 1)); }
    __device__ bool h0(int cc) { return wait(h0r + 8 * (cc & 1), (uint32_t)(cc >> 1) & 1u); }
    __device__ void l1_done() { mma_commit(l1f); }
    __device__ bool h1() { return wait(h1r, 0u); }
    __device__ bool stage(int l, int, int, int akb, uint32_t tcol, bool acc) {
        const int i = k;
        const int s = i % MF_STAGES;
        if (!wait(full0 + 8 * s, (uint32_t)(i / MF_STAGES) & 1u)) return false;
        ++k;
        const uint32_t a = (l == 1 ? r1 : r0) + (uint32_t)akb * MF_KB;
        const uint32_t b = ring + (uint32_t)s * MF_KB;
#pragma unroll
        for (int k16 = 0; k16 < 4; ++k16)
            mma_bf16(tmem + tcol, sw128_desc(a + 32u * k16), sw128_desc(b + 32u * k16), idesc, (acc || k16 > 0) ? 1u : 0u);
        mma_commit(empty0 + 8 * s);
        return true;
    }
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__global__ void __launch_bounds__(MF_THREADS, 1) mlp_fwd_kernel(const __grid_constant__ MlpParams p) {
    extern __shared__ __align__(1024) uint8_t mf_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(mf_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t r0 = smem_u32(smem), r1 = r0 + MF_R0, ring = r1 + MF_R1;
    float* bias_s = reinterpret_cast<float*>(smem + MF_R0 + MF_R1 + MF_STAGES * MF_KB);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + MF_R0 + MF_R1 + MF_STAGES * MF_KB + MF_BIAS);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * MF_STAGES;
    const uint32_t xfull = empty0 + 8 * MF_STAGES, accf = xfull + 8, acce = accf + 16, h0r = acce + 16;
    const uint32_t l1f = h0r + 16, h1r = l1f + 8, drain = h1r + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * MF_STAGES + 11);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* consumed = reinterpret_cast<volatile int*>(tmem_slot + 2);   // weight blocks the MMA waited for

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int net = blockIdx.y, m0 = blockIdx.x * 128;
    const MfDims d{p.K0 / 64, p.N0 / 128, p.N1 / 128, p.N1 / 64, p.N2 / 128};
    const int total = mf_stages_total(d);

    if (threadIdx.x == 0) {
        for (int s = 0; s < MF_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(xfull, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf + 8 * b, 1);
            mbar_init(acce + 8 * b, MF_EPI_WARPS);
            mbar_init(h0r + 8 * b, 1);
        }
        mbar_init(l1f, 1);
        mbar_init(h1r, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    MfProducer pr{&p, net, lane, 0, 0, total, total, ring, full0, empty0, abort_flag};
    // weights that no kernel in flight writes (b_early): the first ring's worth goes out before the wait
    if (p.b_early && warp == 0 && lane < MF_PROD) {
        pr.lo = 0;
        pr.hi = MF_STAGES;
        mf_walk(d, pr);
    }
    // set-up done: wait for the preceding kernel's results (X), let the next kernel's CTAs be placed
    pdl_wait();
    pdl_trigger();

    if (warp == 0) {
        if (lane < MF_PROD) {
            // ---------------- TMA producer: the X tile (lane 0), then the weight blocks
            if (lane == 0) {
                mbar_expect_tx(xfull, (uint32_t)(d.kb0 * MF_KB));
                for (int kb = 0; kb < d.kb0; ++kb) tma_load_2d(r0 + (uint32_t)kb * MF_KB, &p.tmX, xfull, 64 * kb, m0);
            }
            pr.k = 0;
            pr.lo = p.b_early ? MF_STAGES : 0;
            pr.hi = total;
            mf_walk(d, pr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            MfMma mm{tmem, ring, r0, r1, idesc_bf16<128, false, false>(), full0, empty0, accf, acce, h0r, l1f, h1r, 0,
                     p.status, abort_flag};
            if (mm.wait(xfull, 0u)) mf_walk(d, mm);
            *consumed = mm.k;
            // every MMA issued has finished before the TMEM is freed
            mma_commit(drain);
            mbar_wait(drain, 0u, p.status);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: 16 warps, rows 32 q + lane, columns 32 sl .. + 32 of each chunk
        const int e = threadIdx.x - 64, q = warp & 3, sl = (warp - 2) >> 2;
        const int row = 32 * q + lane;
        bool ok = true;
        auto wait_epi = [&](uint32_t bar, uint32_t par) {
            if (!ok) return false;
            if (!mbar_wait(bar, par, p.status, abort_flag)) {
                *abort_flag = 1;
                ok = false;
                return false;
            }
            tc_fence_after();
            return true;
        };
        // one 128-column TMEM chunk (column tcol) -> bias + ELU -> bf16, into K blocks dlo (columns
        // 0-63) and dhi (64-127) of a 128-byte-swizzled region (16-byte unit u of row r at u ^ (r mod 8))
        auto chunk_out = [&](uint32_t tcol, const float* bias, uint32_t dlo, uint32_t dhi, uint32_t rel) {
            uint32_t v[32];
            __syncwarp();
            tmem_ld32_issue(tmem + ((uint32_t)(32 * q) << 16) + tcol + 32u * (uint32_t)sl, v);
            tmem_ld_wait(v);
            if (rel) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(rel);
            }
            float f[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]);
            const float4* b4 = reinterpret_cast<const float4*>(bias + 32 * sl);
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4) {
                const float4 bb = b4[j4];
                elu_bias2(f[4 * j4 + 0], f[4 * j4 + 1], bb.x, bb.y);
                elu_bias2(f[4 * j4 + 2], f[4 * j4 + 3], bb.z, bb.w);
            }
            uint32_t o[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) o[j] = pack_bf16x2(f[2 * j], f[2 * j + 1]);
            const uint32_t dst = (sl < 2 ? dlo : dhi) + (uint32_t)row * 128u;
            const int u0 = (sl & 1) * 4;
#pragma unroll
            for (int g = 0; g < 4; ++g)
                st_shared_v4(dst + ((uint32_t)((u0 + g) ^ (row & 7)) << 4), o[4 * g], o[4 * g + 1], o[4 * g + 2], o[4 * g + 3]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        };
        // the biases (written by the optimiser: read after the wait)
        for (int i = e; i < p.N0 + p.N1 + p.N2; i += 32 * MF_EPI_WARPS)
            bias_s[i] = i < p.N0 ? p.bias[net][0][i] : i < p.N0 + p.N1 ? p.bias[net][1][i - p.N0] : p.bias[net][2][i - p.N0 - p.N1];
        epi_sync();
        const bool store = p.store_hidden != 0;
        // layer 0: chunk c -> H_0 K blocks 2c, 2c + 1 (ring slots mod 4)
        for (int c = 0; c < d.c0; ++c) {
            const bool got = wait_epi(accf + 8 * (c & 1), (uint32_t)(c >> 1) & 1u);
            if (store && c >= 2) {
                if (e == 0) bulk_wait_read<1>();        // chunk c - 2's stores have read its slots
                epi_sync();
            }
            const uint32_t slo = r1 + (uint32_t)((2 * c) & 3) * MF_KB, shi = r1 + (uint32_t)((2 * c + 1) & 3) * MF_KB;
            if (got) chunk_out((uint32_t)(c & 1) * 128u, bias_s + 128 * c, slo, shi, acce + 8 * (c & 1));
            epi_sync();
            if (e == 0 && !*abort_flag) {
                if (store) {
                    tma_store_2d(&p.tmH[net][0], slo, 128 * c, m0);
                    tma_store_2d(&p.tmH[net][0], shi, 128 * c + 64, m0);
                    bulk_commit();
                }
                mbar_arrive(h0r + 8 * (c & 1));
            }
        }
        // layer 1: both halves -> H_1 K blocks in R0 (X is dead: every layer-0 product has completed)
        {
            const bool got = wait_epi(l1f, 0u);
            for (int h = 0; h < d.h1; ++h)
                if (got)
                    chunk_out(256u + 128u * (uint32_t)h, bias_s + p.N0 + 128 * h, r0 + (uint32_t)(2 * h) * MF_KB,
                              r0 + (uint32_t)(2 * h + 1) * MF_KB, 0u);
            epi_sync();
            if (e == 0 && !*abort_flag) {
                if (store) {
                    for (int kb = 0; kb < 2 * d.h1; ++kb) tma_store_2d(&p.tmH[net][1], r0 + (uint32_t)kb * MF_KB, 64 * kb, m0);
                    bulk_commit();
                }
                mbar_arrive(h1r);
            }
        }
        // layer 2: chunk c2 -> H_2 K blocks 2 c2, 2 c2 + 1 in R1 (H_0 is dead: every layer-1 product
        // has completed), out by TMA store
        for (int c2 = 0; c2 < d.c2; ++c2) {
            const int j = d.c0 + c2;
            const bool got = wait_epi(accf + 8 * (j & 1), (uint32_t)(j >> 1) & 1u);
            if (store && c2 == 0) {
                if (e == 0) bulk_wait_read<0>();        // the H_0 stores have read the ring
                epi_sync();
            }
            const uint32_t dlo = r1 + (uint32_t)(2 * c2) * MF_KB, dhi = r1 + (uint32_t)(2 * c2 + 1) * MF_KB;
            if (got) chunk_out((uint32_t)(j & 1) * 128u, bias_s + p.N0 + p.N1 + 128 * c2, dlo, dhi, acce + 8 * (j & 1));
            epi_sync();
            if (e == 0 && !*abort_flag) {
                tma_store_2d(&p.tmH[net][2], dlo, 128 * c2, m0);
                tma_store_2d(&p.tmH[net][2], dhi, 128 * c2 + 64, m0);
                bulk_commit();
            }
        }
        if (e == 0) bulk_wait_all();
    }
    __syncthreads();
    if (warp == 0 && lane < MF_PROD) {
        // copies the MMA never waited for (after a timeout) land before the CTA leaves: at most one
        // per ring slot, the last issued into it
        const int c0 = *consumed;
        for (int i = c0 + ((lane - c0 % MF_PROD) + MF_PROD) % MF_PROD; i < pr.stop; i += MF_PROD)
            mbar_wait(full0 + 8 * (i % MF_STAGES), (uint32_t)(i / MF_STAGES) & 1u, p.status);
        if (lane == 0) mbar_wait(xfull, 0u, p.status);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

}  // namespace

bool mlp_fwd_fits(int K0, int N0, int N1, int N2) {
    return K0 >= 64 && K0 <= 256 && K0 % 64 == 0 && N0 >= 128 && N0 <= 512 && N0 % 128 == 0 && N1 >= 128 && N1 <= 256 &&
           N1 % 128 == 0 && N2 >= 128 && N2 <= 256 && N2 % 128 == 0;
}

cudaError_t mlp_prepare() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MF_SMEM);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

cudaError_t launch_mlp_fwd(const MlpParams& p, cudaStream_t s) {
    if (p.M < 1 || p.nnets < 1 || p.nnets > 2 || !mlp_fwd_fits(p.K0, p.N0, p.N1, p.N2)) return cudaErrorInvalidValue;
    return launch_pdl(mlp_fwd_kernel, dim3((unsigned)((p.M + 127) / 128), (unsigned)p.nnets), dim3(MF_THREADS), (size_t)MF_SMEM, s, p);
}

}  // namespace rl
