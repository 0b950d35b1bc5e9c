// BF16 tensor-core GEMM for the actor/critic MLPs on sm_103a: tcgen05.mma with the FP32
// accumulator in tensor memory, operands staged by TMA into 128-byte-swizzled shared memory,
// and the layer epilogues (bias + ELU, ELU derivative + bias-gradient column sums, split-K
// FP32 partials) fused into the TMEM read-back.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]     A: [M][K] bf16, B: [N][K] bf16, both K contiguous
//
// The MLP products map onto it as
//   forward  H_l = ELU(H_{l-1} W_l^T + b_l):    A = H_{l-1} [rows][in],  B = W_l [out][in]
//   input    dY_{l-1} = (dY_l W_l) * ELU'(H):   A = dY_l [rows][out],    B^T = W_l [out][in]
//   weight   dW_l = dY_l^T H_{l-1}:             A^T = dY_l [rows][out],  B^T = H_{l-1} [rows][in]
// where a transposed operand is read MN-major (the tensor-core descriptors take either form), so
// every operand is used as it is stored and no transposed copy of any matrix is kept.
//
// Persistent CTA per SM, 576 threads, 128 x BN output tiles, K in steps of 64 (one 128-byte
// swizzle row).  warp 0 lane 0 issues TMA loads into a ring of as many stages as fit (full/empty
// mbarriers); warp 1 lane 0 issues 4 tcgen05.mma (K = 16 each) per stage, releases the stage with
// tcgen05.commit and signals a finished tile on one of up to four TMEM accumulators; sixteen
// epilogue warps read the tile back with tcgen05.ld and release the accumulator at once, while the
// next tile accumulates in another.  Every mbarrier wait
// is bounded by the global timer; a wait that runs out records RL_ERR_TIMEOUT in the status
// word, the CTA stops issuing work, waits (bounded) for its copies and MMAs in flight, frees its
// tensor memory and returns.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "gemm_tc.cuh"
#include "tc_prims.cuh"

namespace rl {

namespace {

constexpr int EPI_WARPS = 16;                      // epilogue warps (four per TMEM lane quarter)
constexpr int TC_THREADS = 64 + 32 * EPI_WARPS;    // warp 0: TMA, warp 1: MMA + TMEM owner
constexpr int BM = 128, BK = 64;
constexpr int PROD_LANES = 4;                      // producer lanes of the weight-stationary form
constexpr unsigned PROD_MASK = (1u << PROD_LANES) - 1u;

template <int BN, int EPI, int BROWS = BN, int KS = 1>
struct TileCfg {
    static constexpr int A_BYTES = BM * BK * 2;             // one K block of A
    static constexpr int B_BYTES = BROWS * BK * 2;          // B rows staged per CTA (BN / 2 in pair mode)
    // a stage holds KS K blocks: all of A's, then all of B's
    static constexpr int STAGE = KS * (A_BYTES + B_BYTES);
    // column slices per TMEM lane quarter (4 warps each; fewer slices leave warps idle)
    static constexpr int SLICES = BN / 32 < 4 ? BN / 32 : 4;
    static constexpr int SLICE_COLS = BN / SLICES;
    // per epilogue warp, output blocks leave by TMA store from shared memory: the forward form
    // one 2 KB bf16 block of 32 x 32 (64-byte swizzle), the ELU-gradient form two (it first loads
    // its activation block into the same buffer, one chunk ahead), the fp32 split-K form one 2 KB
    // half block of 32 x 16 at a time (64-byte swizzle)
    static constexpr int STG_WARP = EPI == EPI_ELU_GRAD ? 4096 : 2048;
    static constexpr int STG_BYTES = EPI_WARPS * STG_WARP;
    // the bias is read through L1 (broadcast loads), so that the ring keeps the room
    static constexpr int BIAS_BYTES = 0;
    static constexpr int BAR_BYTES = 512;
    static constexpr int FIXED = STG_BYTES + BIAS_BYTES + BAR_BYTES + 1024 /*align*/;
    // as many ring stages as fit (at most 8): the ring is bound by the copy-to-release turnaround of
    // a stage, so the bytes in flight set its rate
    static constexpr int FIT = (227 * 1024 - FIXED) / STAGE;
    static constexpr int STAGES = FIT > 8 ? 8 : FIT < 2 ? 2 : FIT;
    // TMEM accumulator buffers (BN columns each, 512 columns in all): the MMA warp can run that many
    // tiles ahead of the epilogue
    static constexpr int NACC = 512 / BN < 4 ? 512 / BN : 4;
    static constexpr int SMEM = STAGES * STAGE + FIXED;
};

// Weight-stationary layout (tile mode WS, single CTA): the epilogue's staging blocks and a 1 KB
// barrier block first, then a ring of A stages of two K blocks each (one 3D copy per stage), then
// the CTA's resident B slice (kblocks x BN rows x 128 bytes, sized at run time), with as many ring
// stages as fit (at most 8) in the largest dynamic shared memory of a block.
template <int BN, int EPI>
struct WsCfg {
    using C = TileCfg<BN, EPI>;
    static constexpr int A_STAGE = 2 * C::A_BYTES;
    static constexpr int FRONT = C::STG_BYTES + 1024;
    static constexpr int SMEM = 227 * 1024;
    static constexpr int USABLE = SMEM - 1024;              // after aligning the base to 1 KB
    __host__ __device__ static constexpr int stages(int kblocks) {
        return (USABLE - FRONT - kblocks * BN * 128) / A_STAGE > 8 ? 8 : (USABLE - FRONT - kblocks * BN * 128) / A_STAGE;
    }
};

// The tile sequence of one persistent CTA, t = t0, t0 + step, ..., with each index decoded as
// t = tm + mct (ni + nt (sp + splits b)) (cluster row tile, column tile, split, batch entry).  The
// first index is divided out once; every step then adds the step's own decode with carries, so a
// tile costs the producer and the MMA issuer (single threads, on the pipeline's critical path) a
// few integer adds instead of a chain of divisions by runtime values.
struct TileStep {
    int step, mct, nt, splits, dm, dr;    // dm, dr: step % mct, step / mct
};
struct TileSeq {
    int t, tm, ni, sp, b;
    __device__ TileSeq(int t0, const TileStep& st) {
        t = t0;
        tm = t0 % st.mct;
        int r = t0 / st.mct;
        ni = r % st.nt;
        r /= st.nt;
        sp = r % st.splits;
        b = r / st.splits;
    }
    __device__ void next(const TileStep& st) {
        t += st.step;
        tm += st.dm;
        int c = st.dr;
        if (tm >= st.mct) {
            tm -= st.mct;
            ++c;
        }
        ni += c;
        while (ni >= st.nt) {
            ni -= st.nt;
            if (++sp == st.splits) {
                sp = 0;
                ++b;
            }
        }
    }
};

// Persistent, warp-specialised GEMM.  Output tiles are dealt round-robin to the persistent CTAs
// (one per SM).  In pair mode (PAIR, clusters of CM = 2) two vertically adjacent 128 x BN tiles
// form one 256-row tile on the cta_group::2 tensor core: CTA r of the pair computes row tile
// 2 i + r, loads its own A rows and half of the B tile into its own shared memory, and the even
// CTA issues the MMAs, whose completion arrives on both CTAs' barriers.  No TMA copy is
// multicast.  The TMA warp streams K blocks through a STAGES-deep ring; the MMA warp
// accumulates each tile into one of NACC TMEM buffers (NACC x BN = 512 columns, at most 4 buffers)
// while the sixteen epilogue
// warps drain the other, so the epilogue of tile i overlaps the MMAs of tile i + 1.  Epilogue
// warp e reads TMEM lanes 32 (warp % 4) .. + 31 (its rows) and one slice of up to 4 of the columns.
//
// KS = 2 (single CTA, BN <= 128): a stage carries two K blocks, fetched with one 3D copy per
// operand, and the MMA warp issues eight MMAs per stage wait.  Each TMA copy and each stage
// hand-off costs the issuing thread a fixed few hundred cycles whatever its size, so halving their
// number per K block lifts the narrow tiles' mainloop, which is bound by that per-stage cost rather
// than by the tensor core.  A split or tile with an odd number of K blocks loads a whole last
// stage and multiplies only its first half.
template <int BN, int EPI, int CM, int MJ, bool PAIR, int KS, bool WS = false, bool SR = false>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
    // PAIR: the cluster's two CTAs run one 256 x BN tile on the pair (cta_group::2) tensor core;
    // each CTA stages its 128 rows of A and half of B, the even CTA issues the MMAs
    static_assert(PAIR ? CM == 2 : CM == 1, "clusters of two run the pair MMA only; every other tile is one CTA's");
    static_assert(KS == 1 || (KS == 2 && CM == 1 && !PAIR && BN <= 128), "two-block stages: single CTA, BN <= 128");
    static_assert(!WS || (CM == 1 && !PAIR && KS == 1 && MJ != MAJ_MN && EPI != EPI_STORE),
                  "weight-stationary: single CTA, K-major A, forward or input-gradient epilogue");
    // SR: split-K reduction in a cluster.  Each CTA computes one tile; the p.sred CTAs of a cluster
    // hold consecutive splits of the same tile, stage their fp32 partials in their own (idle) ring
    // memory, and after a cluster barrier each sums a share of the tile's rows over the cluster's
    // partials in rank order, writing one partial per cluster (split group) to p.sr_out.
    static_assert(!SR || (EPI == EPI_STORE && CM == 1 && !PAIR && !WS), "split reduction: split-K partials, single CTA");
    static_assert(!SR || TileCfg<BN, EPI, BN, KS>::STAGES * TileCfg<BN, EPI, BN, KS>::STAGE >= BM * (BN + 4) * 4,
                  "the ring holds a padded fp32 tile");
    using C = TileCfg<BN, EPI, PAIR ? BN / 2 : BN, KS>;
    constexpr bool A_MN = MJ == MAJ_MN;                     // A^T [K][M] in memory
    constexpr bool B_MN = MJ != MAJ_K;                      // B^T [K][N] in memory
    constexpr int B_SLICE_ROWS = PAIR ? BN / 2 : BN / CM;   // B rows this CTA loads
    constexpr int B_BOXES = B_MN ? B_SLICE_ROWS / 64 : 1;   // MN-major: 64-wide boxes per CTA
    static_assert(!B_MN || B_SLICE_ROWS % 64 == 0, "MN-major B tile must split into whole boxes");
    constexpr uint16_t MC_MASK = (uint16_t)((1u << CM) - 1u);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    using W = WsCfg<BN, EPI>;
    // ring stages (run-time in WS mode, where the resident B slice takes its share first)
    const int NS = WS ? W::stages(p.kblocks) : C::STAGES;
    constexpr int NSMAX = WS ? 8 : C::STAGES;               // barrier slots per ring role
    uint8_t* stage_t = WS ? smem : smem + C::STAGES * C::STAGE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(WS ? smem + C::STG_BYTES : smem + C::STAGES * C::STAGE + C::STG_BYTES + C::BIAS_BYTES);
    uint8_t* ring = WS ? smem + W::FRONT : smem;             // the operand stages
    uint8_t* bres = ring + (WS ? NS * W::A_STAGE : 0);       // WS: the resident B slice
    (void)bres;
    // barriers: full[S], empty[S], tfull[NACC], tempty[NACC], drain, bfull (WS: the B slice) (the
    // area keeps room for 2 EPI_WARPS more)
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NSMAX);
    constexpr int NACC = C::NACC;
    const uint32_t tfull0 = smem_u32(bars + 2 * NSMAX), tempty0 = smem_u32(bars + 2 * NSMAX + NACC);
    const uint32_t drain = smem_u32(bars + 2 * NSMAX + 2 * NACC);
    const uint32_t bfull = drain + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSMAX + 2 * NACC + 2 + 2 * EPI_WARPS);
    static_assert((2 * NSMAX + 2 * NACC + 2 + 2 * EPI_WARPS) * 8 + 8 <= (WS ? 1024 : C::BAR_BYTES), "barrier area");
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    // a pair instantiation launched without its cluster shape would address a CTA that does not
    // exist: refuse before touching any barrier
    if (CM > 1 && cluster_size() != (uint32_t)CM) {
        if (threadIdx.x == 0) set_status(p.status, RL_ERR_STATE);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = (p.M + BM - 1) / BM, nt = p.N / BN;
    const int mct = (mt + CM - 1) / CM;                     // cluster tiles along M
    const int total = mct * nt * p.splits * p.batch;
    const int rank = CM > 1 ? (int)cluster_rank() : 0;
    const int cid = CM > 1 ? (int)cluster_id_x() : (int)blockIdx.x;
    const int ncl = CM > 1 ? (int)nclusters_x() : (int)gridDim.x;
    const TileStep tstep{ncl, mct, nt, p.splits, ncl % mct, ncl / mct};
    // SR: the CTA's one tile, t = r + sred (tm + mct (ni + nt (sg + SG b))) with r its rank in the
    // cluster and split sg sred + r (ncl = total, so every role's tile loop runs once)
    auto sr_tile = [&](TileSeq& ts) {
        const int sred = p.sred, r = cid % sred;
        int u = cid / sred;
        ts.tm = u % mct;
        u /= mct;
        ts.ni = u % nt;
        u /= nt;
        const int SG = p.splits / sred;
        ts.sp = (u % SG) * sred + r;
        ts.b = u / SG;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, PAIR ? 2 : 1);             // pair: one arrival per CTA (even CTA's)
            mbar_init(empty0 + 8 * s, PAIR ? 1 : CM);
        }
        mbar_init(bfull, 1);
        for (int a = 0; a < NACC; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, PAIR ? 2 * EPI_WARPS : EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        if (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                         "r"((uint32_t)(NACC * BN))
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                         "r"((uint32_t)(NACC * BN))
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (CM > 1) cluster_sync_all();    // both CTAs' barriers exist before the pair's copies and commits land
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if constexpr (WS) {
        // weights that no kernel in flight writes (b_early): the B slice goes out before the wait
        if (p.b_early && warp == 0 && lane < PROD_LANES) {
            const int G = nt * p.batch, gs = ncl / G, g = cid % G, jr = cid / G;
            if (jr < gs && jr < mct) {
                const CUtensorMap* mb = &p.tmB[g / nt];
                if (lane == 0) mbar_expect_tx(bfull, (uint32_t)(p.kblocks * BN * 128));
                for (int kb = lane; kb < p.kblocks; kb += PROD_LANES) {
                    const uint32_t dst = smem_u32(bres + (size_t)kb * BN * 128);
                    if (!B_MN) tma_load_2d(dst, mb, bfull, kb * BK, (g % nt) * BN);
                    else tma_load_3d(dst, mb, bfull, 0, kb * BK, (g % nt) * BN / 64);
                }
            }
        }
    }
    // set-up done: wait for the preceding kernel's results, let the next kernel's CTAs be placed
    pdl_wait();
    pdl_trigger();

    auto kblocks_of = [&](int sp, int& kb0) {
        kb0 = sp * p.kb_per_split;
        const int kb1 = min(p.kblocks, kb0 + p.kb_per_split);
        return kb1 > kb0 ? kb1 - kb0 : 0;
    };

    if (warp == 0) {
        if constexpr (WS) {
            // ---------------- TMA producer, weight-stationary: CTA cid serves the (network, column
            // tile) group g = cid mod G and its row tiles cid / G, cid / G + ncl / G, ...; its B
            // slice (every K block of the group's BN weight rows) is loaded once, spread over the
            // producer lanes, and only A streams through the ring.  Lane 0 waits for each free stage
            // and posts its byte count; the lanes then take the stages' copies in turn, since one
            // thread's copies are served one after the other at a fixed cost each.
            if (lane < PROD_LANES) {
                const int G = nt * p.batch, gs = ncl / G, g = cid % G, jr = cid / G;
                const int ni = g % nt, b = g / nt;
                const CUtensorMap* ma = &p.tmA[b];
                const CUtensorMap* mb = &p.tmB[b];
                const bool has = jr < gs && jr < mct;
                if (has && !p.b_early) {
                    if (lane == 0) mbar_expect_tx(bfull, (uint32_t)(p.kblocks * BN * 128));
                    for (int kb = lane; kb < p.kblocks; kb += PROD_LANES) {
                        const uint32_t dst = smem_u32(bres + (size_t)kb * BN * 128);
                        if (!B_MN) tma_load_2d(dst, mb, bfull, kb * BK, ni * BN);
                        else tma_load_3d(dst, mb, bfull, 0, kb * BK, ni * BN / 64);
                    }
                }
                const int nst = (p.kblocks + 1) / 2;
                int it = 0, s = 0;
                uint32_t ph = 0;
                bool ok = true;
                for (int mi = jr; has && ok && mi < mct; mi += gs) {
                    for (int i = 0; i < nst; ++i, ++it) {
                        int got = 1;
                        if (lane == 0) {
                            got = mbar_wait(empty0 + 8 * s, ph ^ 1u, p.status, abort_flag) ? 1 : 0;
                            if (got) mbar_expect_tx(full0 + 8 * s, (uint32_t)W::A_STAGE);
                        }
                        got = __shfl_sync(PROD_MASK, got, 0);
                        if (!got) {
                            if (lane == 0) *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        // K blocks 2 i, 2 i + 1 of the row tile (a missing second block reads zeros)
                        if (lane == it % PROD_LANES) tma_load_3d(smem_u32(ring + s * W::A_STAGE), ma, full0 + 8 * s, 0, mi * BM, 2 * i);
                        if (++s == NS) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                }
                if (lane == 0 && has && !ok) {
                    // the copies issued land before the CTA leaves (bounded): the B slice and the
                    // last ring stages
                    mbar_wait(bfull, 0u, p.status);
                    for (int k = 1; k <= NS && it - k >= 0; ++k) {
                        const int j = it - k;
                        mbar_wait(full0 + 8 * (j % NS), (uint32_t)(j / NS) & 1u, p.status);
                    }
                }
            }
        } else if (lane == 0) {
            // ---------------- TMA producer
            int it = 0;
            bool ok = true;
            TileSeq ts0(cid, tstep);
            if (SR) sr_tile(ts0);
            for (TileSeq ts = ts0; ts.t < total && ok; ts.next(tstep)) {
                const int mi = ts.tm * CM + rank, ni = ts.ni, sp = ts.sp, b = ts.b;
                int kb0;
                const int nkb = kblocks_of(sp, kb0);
                const CUtensorMap* ma = &p.tmA[b];
                const CUtensorMap* mb = &p.tmB[b];
                // a row tile past M (the last cluster tile of a ragged M) reloads the last valid
                // rows; its results are never stored
                const int ay = min(mi, mt - 1) * BM;
                const int nst = (nkb + KS - 1) / KS;     // stages of this tile
                for (int i = 0; i < nst; ++i, ++it) {
                    const int s = it % C::STAGES;
                    const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
                    if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.status, abort_flag)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    const uint32_t sa = smem_u32(ring + s * C::STAGE);
                    if constexpr (KS == 2) {
                        // K blocks kb, kb + 1: K-major operands as two 64-column chunks of their rows,
                        // MN-major ones as 128 K rows of their 64-wide M / N chunks
                        const int kb = kb0 + 2 * i;
                        mbar_expect_tx(full0 + 8 * s, (uint32_t)C::STAGE);
                        if (!A_MN) tma_load_3d(sa, ma, full0 + 8 * s, 0, ay, kb);
                        else tma_load_3d(sa, ma, full0 + 8 * s, 0, kb * BK, ay / 64);
                        if (!B_MN) tma_load_3d(sa + 2 * C::A_BYTES, mb, full0 + 8 * s, 0, ni * BN, kb);
                        else tma_load_3d(sa + 2 * C::A_BYTES, mb, full0 + 8 * s, 0, kb * BK, ni * BN / 64);
                        continue;
                    }
                    if constexpr (PAIR) {
                        // both CTAs' copies complete on the even CTA's barrier, which the MMA waits on
                        const uint32_t cfull = mapa_rank(full0 + 8 * s, 0);
                        mbar_expect_tx_cluster(cfull, (uint32_t)C::STAGE);
                        if (!A_MN) {
                            tma_load_2d_pair(sa, ma, cfull, (kb0 + i) * BK, ay);
                        } else {
                            tma_load_2d_pair(sa, ma, cfull, ay, (kb0 + i) * BK);
                            tma_load_2d_pair(sa + 8192, ma, cfull, ay + 64, (kb0 + i) * BK);
                        }
                        if (!B_MN) {
                            tma_load_2d_pair(sa + C::A_BYTES, mb, cfull, (kb0 + i) * BK, ni * BN + rank * B_SLICE_ROWS);
                        } else {
#pragma unroll
                            for (int j = 0; j < B_BOXES; ++j)
                                tma_load_2d_pair(sa + C::A_BYTES + 8192 * j, mb, cfull, ni * BN + rank * B_SLICE_ROWS + 64 * j,
                                                 (kb0 + i) * BK);
                        }
                        continue;
                    }
                    mbar_expect_tx(full0 + 8 * s, (uint32_t)C::STAGE);
                    // single CTA with 3D maps of the MN-major operands: one copy per operand
                    const bool mn3 = CM == 1 && p.mn3;
                    if (!A_MN) {
                        tma_load_2d(sa, ma, full0 + 8 * s, (kb0 + i) * BK, ay);
                    } else if (mn3) {
                        tma_load_3d(sa, ma, full0 + 8 * s, 0, (kb0 + i) * BK, ay / 64);
                    } else {
                        // [K][M] source: two boxes of 64 M columns x 64 K rows
                        tma_load_2d(sa, ma, full0 + 8 * s, ay, (kb0 + i) * BK);
                        tma_load_2d(sa + 8192, ma, full0 + 8 * s, ay + 64, (kb0 + i) * BK);
                    }
                    if (!B_MN) {
                        tma_load_2d(sa + C::A_BYTES, mb, full0 + 8 * s, (kb0 + i) * BK, ni * BN);
                    } else if (mn3) {
                        tma_load_3d(sa + C::A_BYTES, mb, full0 + 8 * s, 0, (kb0 + i) * BK, ni * BN / 64);
                    } else {
                        // [K][N] source: boxes of 64 N columns x 64 K rows
#pragma unroll
                        for (int j = 0; j < B_BOXES; ++j)
                            tma_load_2d(sa + C::A_BYTES + 8192 * j, mb, full0 + 8 * s, ni * BN + 64 * j, (kb0 + i) * BK);
                    }
                }
            }
            if (!ok && !PAIR) {
                // let the copies already issued land before the CTA leaves (bounded; in pair mode
                // they complete on the even CTA's barriers and cannot be observed here)
                for (int k = 1; k <= C::STAGES && it - k >= 0; ++k) {
                    const int j = it - k;
                    mbar_wait(full0 + 8 * (j % C::STAGES), (uint32_t)(j / C::STAGES) & 1u, p.status);
                }
            } else if (ok && CM > 1) {
                // every CTA of the cluster has released the last use of each stage: no copy or
                // MMA-completion arrival of this cluster can still target this CTA's memory
                for (int k = 1; k <= C::STAGES && it - k >= 0; ++k) {
                    const int j = it - k;
                    if (!mbar_wait(empty0 + 8 * (j % C::STAGES), (uint32_t)(j / C::STAGES) & 1u, p.status)) break;
                }
            }
        }
    } else if (warp == 1) {
        if (WS && lane == 0) {
            // ---------------- MMA issuer, weight-stationary: A from the ring, B from the resident
            // slice; eight MMAs (two K blocks) per stage hand-off
            const uint32_t idesc = idesc_bf16<BN, false, B_MN>();
            const int G = nt * p.batch, gs = ncl / G, jr = cid / G;
            const uint64_t ad0 = sw128_desc(smem_u32(ring));
            const uint64_t bd0 = B_MN ? sw128_desc_mn(smem_u32(bres), 8192u) : sw128_desc(smem_u32(bres));
            constexpr uint64_t KSTEP_B = B_MN ? (2048 >> 4) : (32 >> 4);
            constexpr uint64_t BKB = (uint64_t)(BN * 128) >> 4;      // one K block of the resident B
            constexpr uint64_t ASUB = (uint64_t)C::A_BYTES >> 4;     // the stage's second K block
            const int nst = (p.kblocks + 1) / 2;
            const bool has = jr < gs && jr < mct;
            bool ok = !has || mbar_wait(bfull, 0u, p.status, abort_flag);
            if (!ok) *abort_flag = 1;
            int local = 0, s = 0;
            uint32_t ph = 0;
            for (int mi = jr; has && ok && mi < mct; mi += gs, ++local) {
                const int a = local % NACC;
                const uint32_t aph = (uint32_t)(local / NACC) & 1u;
                if (!mbar_wait(tempty0 + 8 * a, aph ^ 1u, p.status, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * BN);
                for (int i = 0; i < nst; ++i) {
                    if (!mbar_wait(full0 + 8 * s, ph, p.status, abort_flag)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = ad0 + (uint64_t)((s * W::A_STAGE) >> 4);
                    const int nsub = min(2, p.kblocks - 2 * i);
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        if (j >= nsub) break;
                        const uint64_t bd = bd0 + BKB * (uint64_t)(2 * i + j);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_bf16(d, ad + ASUB * j + 2 * kk, bd + KSTEP_B * kk, idesc, (i > 0 || j > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(empty0 + 8 * s);
                    if (++s == NS) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(tfull0 + 8 * a);
            }
            // drain: every MMA issued has finished before the TMEM is freed
            mma_commit(drain);
            mbar_wait(drain, 0u, p.status);
        } else if (!WS && lane == 0) {
            // ---------------- MMA issuer (pair mode: the even CTA only)
            const uint32_t idesc = idesc_bf16<BN, A_MN, B_MN, PAIR ? 2 * BM : BM>();
            int it = 0, local = 0;
            bool ok = true;
            const bool issuer = !PAIR || rank == 0;
            const uint32_t sa0 = smem_u32(ring);
            constexpr uint32_t LBO = KS == 2 ? 16384u : 8192u;   // MN-major: bytes between 64-wide chunks
            const uint64_t ad0 = A_MN ? sw128_desc_mn(sa0, LBO) : sw128_desc(sa0);
            const uint64_t bd0 = B_MN ? sw128_desc_mn(sa0 + KS * C::A_BYTES, LBO) : sw128_desc(sa0 + KS * C::A_BYTES);
            TileSeq ts0(cid, tstep);
            if (SR) sr_tile(ts0);
            for (TileSeq ts = ts0; issuer && ts.t < total && ok; ts.next(tstep), ++local) {
                int kb0;
                const int nkb = kblocks_of(ts.sp, kb0);
                const int a = local % NACC;
                const uint32_t aph = (uint32_t)(local / NACC) & 1u;
                if (!mbar_wait(tempty0 + 8 * a, aph ^ 1u, p.status, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * BN);
                const int nst = (nkb + KS - 1) / KS;
                for (int i = 0; i < nst; ++i, ++it) {
                    const int s = it % C::STAGES;
                    const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
                    if (!mbar_wait(full0 + 8 * s, ph, p.status, abort_flag)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // stage s descriptors: stage 0's plus the stage offset in 16-byte units
                    const uint64_t soff = (uint64_t)((s * C::STAGE) >> 4);
                    const uint64_t ad = ad0 + soff, bd = bd0 + soff;
                    // K16 step: 32 bytes along the swizzled row (K-major), two 8-row atoms (MN-major)
                    constexpr uint64_t KSTEP_A = A_MN ? (2048 >> 4) : (32 >> 4);
                    constexpr uint64_t KSTEP_B = B_MN ? (2048 >> 4) : (32 >> 4);
                    if constexpr (KS == 2) {
                        // second K block: 64 K rows further (MN-major), the next chunk (K-major)
                        constexpr uint64_t SUB_A = A_MN ? (8192 >> 4) : (C::A_BYTES >> 4);
                        constexpr uint64_t SUB_B = B_MN ? (8192 >> 4) : (C::B_BYTES >> 4);
                        const int nsub = min(2, nkb - 2 * i);
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            if (j >= nsub) break;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk)
                                mma_bf16(d, ad + SUB_A * j + KSTEP_A * kk, bd + SUB_B * j + KSTEP_B * kk, idesc,
                                         (i > 0 || j > 0 || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(empty0 + 8 * s);
                    } else if constexpr (PAIR) {
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_bf16_pair(d, ad + KSTEP_A * kk, bd + KSTEP_B * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                        mma_commit_pair_mc(empty0 + 8 * s, MC_MASK);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_bf16(d, ad + KSTEP_A * kk, bd + KSTEP_B * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(empty0 + 8 * s);
                    }
                }
                // arrives when every MMA issued so far has completed (pair: in both CTAs)
                if constexpr (PAIR) mma_commit_pair_mc(tfull0 + 8 * a, MC_MASK);
                else mma_commit(tfull0 + 8 * a);
            }
            if (issuer) {
                // drain: every MMA this thread issued has finished before the TMEM is freed
                if constexpr (PAIR) mma_commit_pair(drain);
                else mma_commit(drain);
                mbar_wait(drain, 0u, p.status);
                if (PAIR && ok && !*abort_flag) {
                    // the odd CTA's epilogue arrives on this CTA's tempty barriers: wait for the last
                    // release of each buffer so that no arrival is still on its way when this CTA leaves
                    for (int k = 1; k <= NACC && local - k >= 0; ++k) {
                        const int j = local - k;
                        if (!mbar_wait(tempty0 + 8 * (j % NACC), (uint32_t)(j / NACC) & 1u, p.status)) break;
                    }
                }
            }
        }
    } else {
        // ---------------- epilogue warps
        const int ew = warp - 2;
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int slice = ew >> 2;              // column slice of the tile (slice >= SLICES: idle)
        const bool busy = slice < C::SLICES;
        uint8_t* stg_raw = stage_t + (size_t)ew * C::STG_WARP;
        // ELU-gradient form: the warp's activation blocks (32 rows x 32 columns of H per chunk) are
        // fetched by cp.async (four lanes per 64-byte row, rows past M read as zeros) into two
        // buffers with the output block's swizzle, one chunk ahead of the chunk being processed;
        // the load/store unit carries them so that the TMA unit serves only the operand stream and
        // the output stores
        constexpr int CPT = C::SLICE_COLS / 32;                 // chunks per tile of one warp
        constexpr int PRE = EPI == EPI_ELU_GRAD ? 1 : CPT;      // chunks loaded from TMEM together
        int hj = 0;                                              // chunks processed so far
        // the epilogue warps decode each tile by division: the latency is theirs alone and other
        // warps cover it, and the incremental form's extra live registers would spill here
        auto decode = [&](int t, int& mi, int& ni, int& sp, int& b) {
            mi = (t % mct) * CM + rank;
            int r = t / mct;
            ni = r % nt;
            r /= nt;
            sp = r % p.splits;
            b = r / p.splits;
        };
        // the k-th tile of this CTA (false past its last): tile cid + k ncl of the global order, or
        // in WS mode row tile cid / G + k ncl / G of its group (network, column tile) cid mod G
        auto tile_at = [&](int k, int& mi, int& ni, int& sp, int& b) -> bool {
            if constexpr (WS) {
                const int G = nt * p.batch, gs = ncl / G, g = cid % G;
                mi = cid / G + k * gs;
                ni = g % nt;
                b = g / nt;
                sp = 0;
                return cid / G < gs && mi < mct;
            } else {
                const int t = cid + k * ncl;
                if (t >= total) return false;
                if (SR) {
                    TileSeq ts(cid, tstep);
                    sr_tile(ts);
                    mi = ts.tm;
                    ni = ts.ni;
                    sp = ts.sp;
                    b = ts.b;
                } else {
                    decode(t, mi, ni, sp, b);
                }
                return true;
            }
        };
        auto h_issue = [&](int j) {
            // chunk j of this warp's sequence: the CTA's tile j / CPT, column chunk j % CPT
            // the output store that last read the buffer (chunk j - 2) is done reading it
            if (lane == 0) bulk_wait_read<0>();
            __syncwarp();
            int mi, ni, sp, b;
            if (tile_at(j / CPT, mi, ni, sp, b)) {
                const int x = ni * BN + slice * C::SLICE_COLS + 32 * (j % CPT);
                const int y = mi * BM + 32 * q;
                const uint32_t dst = smem_u32(stg_raw + 2048 * (j & 1));
                const int u = lane & 3;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = 8 * i + (lane >> 2);
                    const bool ok = y + r < p.M;
                    const __nv_bfloat16* src = reinterpret_cast<const __nv_bfloat16*>(p.hsrc[b]) +
                                               (size_t)(ok ? y + r : 0) * p.ldh + x + 8 * u;
                    cp_async16(dst + r * 64 + 16 * (u ^ ((r >> 1) & 3)), src, ok ? 16u : 0u);
                }
            }
            cp_async_commit();     // an empty group past the last chunk keeps the wait counts uniform
        };
        if (EPI == EPI_ELU_GRAD && busy) h_issue(0);
        int oj = 0;                                              // bf16 output blocks written (buffer index)
        for (int local = 0;; ++local) {
            int mi, ni, sp, b, kb0;
            if (!tile_at(local, mi, ni, sp, b)) break;
            const int nkb = kblocks_of(sp, kb0);
            const int a = local % NACC;
            const uint32_t aph = (uint32_t)(local / NACC) & 1u;
            const int m0 = mi * BM, n0 = ni * BN;
            const int row = m0 + 32 * q + lane;
            const bool row_ok = row < p.M;
            const bool tile_ok = mi < mt;
            if (!mbar_wait(tfull0 + 8 * a, aph, p.status, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            // this warp's columns of the tile leave TMEM at once (the ELU-gradient form, short of
            // registers, loads its chunks one by one) and the accumulator is released before the
            // math and the stores, so the MMAs of a later tile can start in it
            auto tmem_col = [&](int ch) {
                return tmem + (uint32_t)(a * BN) + ((uint32_t)(32 * q) << 16) + (uint32_t)(slice * C::SLICE_COLS + 32 * ch);
            };
            auto release = [&]() {
                // pair: on the even CTA's barrier
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (PAIR) mbar_arrive_cluster(mapa_rank(tempty0 + 8 * a, 0));
                    else mbar_arrive(tempty0 + 8 * a);
                }
            };
            uint32_t r[CPT][32];
            if (busy) {
#pragma unroll
                for (int ch = 0; ch < PRE; ++ch) tmem_ld32_issue(tmem_col(ch), r[ch]);
                tmem_ld_wait(r[0]);
#pragma unroll
                for (int ch = 1; ch < PRE; ++ch) tmem_ld_after_wait(r[ch]);
            }
            if (PRE == CPT || !busy) release();
#pragma unroll
            for (int ch = 0; ch < CPT; ++ch) {
                if (!busy) break;
                if (ch >= PRE) {
                    tmem_ld32_issue(tmem_col(ch), r[ch]);
                    tmem_ld_wait(r[ch]);
                    if (ch == CPT - 1) release();
                }
                const int c = slice * C::SLICE_COLS + 32 * ch;
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[ch][j]);
                if (EPI == EPI_STORE && nkb == 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.f;
                }
                const int col = n0 + c;
                if (EPI == EPI_STORE && SR) {
                    // the partial into this CTA's ring memory, free now that the tile's MMAs are
                    // done: row 32 q + lane, padded rows (BN + 4 floats: 16-byte stores of 8 lanes
                    // meet 32 different banks)
                    float* red = reinterpret_cast<float*>(ring) + (size_t)(32 * q + lane) * (BN + 4) + c;
#pragma unroll
                    for (int j4 = 0; j4 < 8; ++j4)
                        *reinterpret_cast<float4*>(red + 4 * j4) = make_float4(v[4 * j4], v[4 * j4 + 1], v[4 * j4 + 2], v[4 * j4 + 3]);
                } else if (EPI == EPI_STORE) {
                    // two fp32 half blocks of 32 rows x 16 columns through the 2 KB buffer (64-byte
                    // swizzle: 16-byte unit u of row r at unit u ^ ((r >> 1) & 3)), each out by TMA
                    // store once the previous store from the buffer has read it
                    const int sw = (lane >> 1) & 3;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        if (lane == 0) bulk_wait_read<0>();
                        __syncwarp();
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            *reinterpret_cast<float4*>(stg_raw + lane * 64 + 16 * (u ^ sw)) =
                                make_float4(v[16 * hh + 4 * u], v[16 * hh + 4 * u + 1], v[16 * hh + 4 * u + 2],
                                            v[16 * hh + 4 * u + 3]);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0 && tile_ok) {
                            tma_store_3d(&p.tmC[b], smem_u32(stg_raw), col + 16 * hh, m0 + 32 * q, sp);
                            bulk_commit();
                        }
                    }
                } else if (EPI == EPI_BIAS_ELU) {
                    const float4* bias4 = reinterpret_cast<const float4*>(p.bias[b] + col);
#pragma unroll
                    for (int j4 = 0; j4 < 8; ++j4) {
                        const float4 bb = __ldg(bias4 + j4);
                        elu_bias2(v[4 * j4 + 0], v[4 * j4 + 1], bb.x, bb.y);
                        elu_bias2(v[4 * j4 + 2], v[4 * j4 + 3], bb.z, bb.w);
                    }
                    uint32_t o[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) o[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
                    // bf16 block in one of two buffers (64-byte swizzle: 16-byte unit u of row r at
                    // unit u ^ ((r >> 1) & 3)), out by TMA store; the store issued from this buffer
                    // two blocks ago must have read it
                    uint8_t* ob = stg_raw;
                    if (lane == 0) bulk_wait_read<0>();
                    __syncwarp();
                    const int sw = (lane >> 1) & 3;
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        *reinterpret_cast<uint4*>(ob + lane * 64 + 16 * (g ^ sw)) =
                            make_uint4(o[4 * g], o[4 * g + 1], o[4 * g + 2], o[4 * g + 3]);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0 && tile_ok) {
                        tma_store_3d(&p.tmC[b], smem_u32(ob), col, m0 + 32 * q, 0);
                        bulk_commit();
                    }
                    ++oj;
                } else {   // EPI_ELU_GRAD
                    // the next chunk's activations go into the other buffer, then this chunk's
                    // copies (every lane's) are waited for
                    h_issue(hj + 1);
                    uint8_t* hb = stg_raw + 2048 * (hj & 1);
                    cp_async_wait<1>();
                    __syncwarp();
                    // 64-byte swizzle: 16-byte unit u of row r sits at unit u ^ ((r >> 1) & 3)
                    const int sw = (lane >> 1) & 3;
                    if (row_ok) {
                        // ELU'(x) from y = ELU(x): 1 for y > 0, y + 1 otherwise, i.e. min(y, 0) + 1,
                        // so the product is fma(v, min(y, 0), v)
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            const uint4 hv = *reinterpret_cast<const uint4*>(hb + lane * 64 + 16 * (g ^ sw));
                            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float y0 = __uint_as_float(hw[j] << 16), y1 = __uint_as_float(hw[j] & 0xFFFF0000u);
                                const uint64_t vv = f2_pack(v[8 * g + 2 * j], v[8 * g + 2 * j + 1]);
                                f2_unpack(f2_fma(vv, f2_pack(fminf(y0, 0.f), fminf(y1, 0.f)), vv), v[8 * g + 2 * j],
                                          v[8 * g + 2 * j + 1]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = 0.f;
                    }
                    uint32_t o[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) o[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
                    // the output block replaces the activation block in place (same swizzle) and
                    // leaves by TMA store
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        *reinterpret_cast<uint4*>(hb + lane * 64 + 16 * (g ^ sw)) =
                            make_uint4(o[4 * g], o[4 * g + 1], o[4 * g + 2], o[4 * g + 3]);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0 && tile_ok) {
                        tma_store_3d(&p.tmC[b], smem_u32(hb), col, m0 + 32 * q, 0);
                        bulk_commit();
                    }
                    ++hj;
                    if (p.colsum[b]) {
                        const float s = colsum32(v, lane);    // column col + lane, over this warp's 32 rows
                        if (tile_ok) p.colsum[b][((size_t)mi * 4 + q) * p.N + col + lane] = s;
                    }
                }
            }
        }
        // activation copies still in flight land and the output stores complete before the CTA
        // leaves
        if (EPI == EPI_ELU_GRAD) cp_async_wait<0>();
        if (lane == 0) bulk_wait_all();
    }
    if constexpr (SR) {
        // every CTA of the cluster has staged its partial (the barrier orders the shared-memory
        // writes before the peers' reads); CTA r then sums rows [r BM / sred, (r + 1) BM / sred) of
        // the tile over ranks 0 .. sred - 1 in order and writes them to its split group's partial;
        // the second barrier keeps each CTA's memory until the peers have read it
        __syncwarp();
        cluster_sync_all();
        if (warp >= 2) {
            TileSeq ts(cid, tstep);
            sr_tile(ts);
            const int sred = p.sred, r = cid % sred, sg = ts.sp / sred;
            const int r0 = r * BM / sred, r1 = (r + 1) * BM / sred;
            const int m0 = ts.tm * BM, n0 = ts.ni * BN;
            constexpr int C4 = BN / 4;
            const uint32_t red0 = smem_u32(ring);
            float* out = p.sr_out[ts.b] + (size_t)sg * p.sr_split_ld;
            for (int e = threadIdx.x - 64; e < (r1 - r0) * C4; e += 32 * EPI_WARPS) {
                const int row = r0 + e / C4, c4 = e % C4;
                const uint32_t off = (uint32_t)((row * (BN + 4) + 4 * c4) * 4);
                float4 acc = ld_cluster_f4(mapa_rank(red0 + off, 0));
                for (int k = 1; k < sred; ++k) {
                    const float4 x = ld_cluster_f4(mapa_rank(red0 + off, (uint32_t)k));
                    acc.x += x.x;
                    acc.y += x.y;
                    acc.z += x.z;
                    acc.w += x.w;
                }
                if (m0 + row < p.M)
                    *reinterpret_cast<float4*>(out + (size_t)(m0 + row) * p.sr_ld + n0 + 4 * c4) = acc;
            }
        }
        cluster_sync_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        if (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(NACC * BN)) : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(NACC * BN)) : "memory");
    }
}

// Clusters of CM CTAs that fit on the device at once (one CTA per SM), per instantiation;
// measured once in tc_prepare (before any stream capture) and used to size the persistent grid.
struct ClusterFit {
    int clusters[3][3][3];    // [bn 64/128/256][epi][single CTA, weight-stationary, pair]
};
static ClusterFit g_fit[64];

static int bn_index(int bn) { return bn == 64 ? 0 : bn == 128 ? 1 : bn == 256 ? 2 : -1; }
// cluster modes of the ABI: 1 single CTA (and 4, its two-K-block form), 3 the cta_group::2 pair
static int cm_index(int cm) { return cm == 1 || cm == 4 ? 0 : cm == 3 ? 2 : -1; }

template <int BN, int EPI, int CM, int MJ, bool PAIR, int KS, bool WS = false, bool SR = false>
constexpr int smem_of() {
    return WS ? WsCfg<BN, EPI>::SMEM : TileCfg<BN, EPI, PAIR ? BN / 2 : BN, KS>::SMEM;
}
// slot of the cluster-fit table: 0 single CTA, 1 weight-stationary single CTA, 2 pair
template <int CM, bool PAIR, bool WS = false>
constexpr int fit_slot() {
    return PAIR ? 2 : WS ? 1 : 0;
}

template <int BN, int EPI, int CM, int MJ, bool PAIR, int KS = 1, bool WS = false, bool SR = false>
cudaError_t set_attr(int dev) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN, EPI, CM, MJ, PAIR, KS, WS, SR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_of<BN, EPI, CM, MJ, PAIR, KS, WS>());
    if (SR) return e;                    // grid = the tile count; the fit table belongs to the plain forms
    if (e != cudaSuccess) return e;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int n = sms / CM;
    if (CM > 1) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CM;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(n * CM));
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = smem_of<BN, EPI, CM, MJ, PAIR, KS>();
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int fit = 0;
        e = cudaOccupancyMaxActiveClusters(&fit, tc_gemm_kernel<BN, EPI, CM, MJ, PAIR, KS>, &cfg);
        if (e != cudaSuccess) return e;
        if (fit > 0 && fit < n) n = fit;
    }
    if (dev >= 0 && dev < 64) g_fit[dev].clusters[bn_index(BN)][EPI][fit_slot<CM, PAIR, WS>()] = n > 0 ? n : 1;
    return cudaSuccess;
}

template <int BN, int EPI, int CM, int MJ, bool PAIR, int KS = 1, bool WS = false, bool SR = false>
cudaError_t launch_cfg(const TcParams& p, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    int fit = (dev >= 0 && dev < 64) ? g_fit[dev].clusters[bn_index(BN)][EPI][fit_slot<CM, PAIR, WS>()] : 0;
    if (fit <= 0) return cudaErrorNotReady;        // tc_prepare has not run on this device
    const int mct = ((p.M + BM - 1) / BM + CM - 1) / CM;
    const int total = mct * (p.N / BN) * p.splits * p.batch;
    int clusters = total < fit ? total : fit;            // one persistent CTA per SM
    if (p.max_ctas > 0 && clusters > p.max_ctas / CM) clusters = p.max_ctas / CM > 0 ? p.max_ctas / CM : 1;
    constexpr int SMEM = smem_of<BN, EPI, CM, MJ, PAIR, KS, WS>();
    if constexpr (SR) {
        // one CTA per tile and split, clusters of p.sred consecutive splits of one tile
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)p.sred;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.gridDim = dim3((unsigned)total);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = SMEM;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<BN, EPI, 1, MJ, false, KS, false, true>, p);
    }
    if constexpr (WS) {
        // a whole number of CTAs per (network, column tile) group, at least one each (a CTA cap
        // below the group count is raised to it)
        const int G = (p.N / BN) * p.batch;
        if (G > fit) return cudaErrorInvalidValue;
        clusters = clusters < G ? G : clusters / G * G;
        return launch_pdl(tc_gemm_kernel<BN, EPI, 1, MJ, false, 1, true>, dim3(clusters), dim3(TC_THREADS), SMEM, s, p);
    }
    if constexpr (CM == 1) {
        return launch_pdl(tc_gemm_kernel<BN, EPI, 1, MJ, false, KS>, dim3(clusters), dim3(TC_THREADS), SMEM, s, p);
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CM;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3((unsigned)(clusters * CM));
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<BN, EPI, CM, MJ, PAIR, KS>, p);
}

// Instantiated operand forms: forward (EPI_BIAS_ELU) both K-major; input gradient
// (EPI_ELU_GRAD) A K-major, B = W read MN-major; split-K weight gradient and the diagnostic
// GEMMs (EPI_STORE) both K-major or both MN-major.  A cluster of 2 with an MN-major B needs
// whole 64-column boxes per CTA (BN >= 128); pair mode runs with BN = 128 or 256.

template <int BN, int EPI, int MJ>
cudaError_t launch_cm_mj(const TcParams& p, cudaStream_t s) {
    if (p.ws) {
        if constexpr (EPI != EPI_STORE && MJ != MAJ_MN) return launch_cfg<BN, EPI, 1, MJ, false, 1, true>(p, s);
        return cudaErrorInvalidValue;
    }
    if (p.cm == 1 && p.sred >= 1) {
        if constexpr (EPI == EPI_STORE && MJ == MAJ_MN) {
            if (p.ks == 2) {
                if constexpr (BN <= 128) return launch_cfg<BN, EPI, 1, MJ, false, 2, false, true>(p, s);
                return cudaErrorInvalidValue;
            }
            return launch_cfg<BN, EPI, 1, MJ, false, 1, false, true>(p, s);
        }
        return cudaErrorInvalidValue;
    }
    if (p.cm == 1) {
        if (p.ks == 2) {
            if constexpr (BN <= 128) return launch_cfg<BN, EPI, 1, MJ, false, 2>(p, s);
            return cudaErrorInvalidValue;
        }
        return launch_cfg<BN, EPI, 1, MJ, false>(p, s);
    }
    if (p.cm == 2 && p.pair) {
        if constexpr (BN >= 128) return launch_cfg<BN, EPI, 2, MJ, true>(p, s);
    }
    return cudaErrorInvalidValue;
}

template <int BN, int EPI>
cudaError_t launch_cm(const TcParams& p, cudaStream_t s) {
    if constexpr (EPI == EPI_BIAS_ELU) {
        if (p.mn == MAJ_K) return launch_cm_mj<BN, EPI, MAJ_K>(p, s);
    } else if constexpr (EPI == EPI_ELU_GRAD) {
        if (p.mn == MAJ_B_MN) return launch_cm_mj<BN, EPI, MAJ_B_MN>(p, s);
    } else {
        if (p.mn == MAJ_K) return launch_cm_mj<BN, EPI, MAJ_K>(p, s);
        if (p.mn == MAJ_MN) return launch_cm_mj<BN, EPI, MAJ_MN>(p, s);
    }
    return cudaErrorInvalidValue;
}

template <int EPI>
cudaError_t launch_bn(const TcParams& p, cudaStream_t s) {
    switch (p.bn) {
        case 64: return launch_cm<64, EPI>(p, s);
        case 128: return launch_cm<128, EPI>(p, s);
        case 256: return launch_cm<256, EPI>(p, s);
    }
    return cudaErrorInvalidValue;
}

template <int EPI, int MJ>
cudaError_t prepare_form(int dev) {
    cudaError_t e = cudaSuccess;
    e = e != cudaSuccess ? e : set_attr<64, EPI, 1, MJ, false>(dev);
    e = e != cudaSuccess ? e : set_attr<128, EPI, 1, MJ, false>(dev);
    e = e != cudaSuccess ? e : set_attr<256, EPI, 1, MJ, false>(dev);
    e = e != cudaSuccess ? e : set_attr<128, EPI, 2, MJ, true>(dev);
    e = e != cudaSuccess ? e : set_attr<256, EPI, 2, MJ, true>(dev);
    e = e != cudaSuccess ? e : set_attr<64, EPI, 1, MJ, false, 2>(dev);
    e = e != cudaSuccess ? e : set_attr<128, EPI, 1, MJ, false, 2>(dev);
    if constexpr (EPI == EPI_STORE && MJ == MAJ_MN) {
        e = e != cudaSuccess ? e : set_attr<64, EPI, 1, MJ, false, 1, false, true>(dev);
        e = e != cudaSuccess ? e : set_attr<128, EPI, 1, MJ, false, 1, false, true>(dev);
        e = e != cudaSuccess ? e : set_attr<256, EPI, 1, MJ, false, 1, false, true>(dev);
        e = e != cudaSuccess ? e : set_attr<64, EPI, 1, MJ, false, 2, false, true>(dev);
        e = e != cudaSuccess ? e : set_attr<128, EPI, 1, MJ, false, 2, false, true>(dev);
    }
    if constexpr (EPI != EPI_STORE && MJ != MAJ_MN) {
        e = e != cudaSuccess ? e : set_attr<64, EPI, 1, MJ, false, 1, true>(dev);
        e = e != cudaSuccess ? e : set_attr<128, EPI, 1, MJ, false, 1, true>(dev);
        e = e != cudaSuccess ? e : set_attr<256, EPI, 1, MJ, false, 1, true>(dev);
    }
    return e;
}

}  // namespace

cudaError_t launch_tc_gemm(const TcParams& p, cudaStream_t s) {
    if (p.M <= 0) return cudaSuccess;
    if (p.bn <= 0 || p.N % p.bn || p.kblocks <= 0 || p.splits <= 0 || p.batch < 1 || p.batch > 2) return cudaErrorInvalidValue;
    if (p.cm != 1 && p.cm != 2) return cudaErrorInvalidValue;
    if (p.mn != MAJ_K && p.mn != MAJ_MN && p.mn != MAJ_B_MN) return cudaErrorInvalidValue;
    if (p.pair && (p.cm != 2 || p.bn < 128)) return cudaErrorInvalidValue;
    if (p.cm == 2 && !p.pair) return cudaErrorInvalidValue;     // clusters of two run the pair MMA only
    if (p.ks < 0 || p.ks > 2 || (p.ks == 2 && (p.cm != 1 || p.pair || p.bn > 128))) return cudaErrorInvalidValue;
    if (p.mn3 && (p.cm != 1 || p.pair || p.ks == 2 || p.mn == MAJ_K)) return cudaErrorInvalidValue;
    // split reduction in a cluster: split-K partials of both-MN-major operands, single CTA, a cluster
    // size of 1..8 dividing the split count, an output for the cluster partials
    if (p.sred != 0 && (p.sred < 1 || p.sred > 8 || p.splits % p.sred || p.epi != EPI_STORE || p.mn != MAJ_MN || p.cm != 1 ||
                        p.pair || p.ws || !p.sr_out[0] || (p.batch > 1 && !p.sr_out[1]) || p.sr_ld < p.N || p.sr_ld % 4 ||
                        p.sr_split_ld % 4 || (reinterpret_cast<uintptr_t>(p.sr_out[0]) & 15u) ||
                        (p.batch > 1 && (reinterpret_cast<uintptr_t>(p.sr_out[1]) & 15u))))
        return cudaErrorInvalidValue;
    // weight-stationary: single CTA, no split, forward (B K-major) or input gradient (B by the 3D
    // MN-major maps), at least one ring stage beside the resident B slice
    if (p.b_early && !p.ws) return cudaErrorInvalidValue;
    if (p.ws && (p.cm != 1 || p.pair || p.ks == 2 || p.splits != 1 || p.epi == EPI_STORE || (p.mn == MAJ_B_MN && !p.mn3) ||
                 tc_ws_stages(p.bn, p.epi, p.kblocks) < 1))
        return cudaErrorInvalidValue;
    if (p.epi == EPI_ELU_GRAD) {
        // activation rows are read as 16-byte pieces
        for (int b = 0; b < p.batch; ++b)
            if (!p.hsrc[b] || (reinterpret_cast<uintptr_t>(p.hsrc[b]) & 15u)) return cudaErrorInvalidValue;
        if (p.ldh < p.N || p.ldh % 8) return cudaErrorInvalidValue;
    }
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
static bool make_tmap(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_cols,
                      uint32_t box_rows, CUtensorMapSwizzle sw) {
    EncodeTiledFn enc = get_encode();
    if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15u) || (ld * 2) % 16 || cols > ld) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows) {
    return make_tmap(map, base, rows, cols, ld, (uint32_t)BK, box_rows, CU_TENSOR_MAP_SWIZZLE_128B);
}

// bf16 [rows][cols] viewed as {64, rows, cols / 64} (64-element chunks 128 bytes apart), box
// {64, box_rows, box_chunks}, 128-byte swizzle.  cols must be a multiple of 64 so that no chunk
// reaches past a row; chunks of a box past the last one read as zeros.
static bool make_tmap_chunks(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows,
                             uint32_t box_chunks) {
    EncodeTiledFn enc = get_encode();
    if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15u) || (ld * 2) % 16 || cols > ld || cols % 64 ||
        box_rows < 1 || box_rows > 256 || box_chunks < 1 || box_chunks > 4)
        return false;
    cuuint64_t dims[3] = {64, rows, cols / 64};
    cuuint64_t strides[2] = {ld * 2, 128};
    cuuint32_t box[3] = {64, box_rows, box_chunks};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_tmap_bf16_k2(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows) {
    return make_tmap_chunks(map, base, rows, cols, ld, box_rows, 2);
}

bool make_tmap_bf16_mn2(CUtensorMap* map, const void* base, uint64_t krows, uint64_t cols, uint64_t ld, uint32_t tile_cols) {
    return tile_cols % 64 == 0 && make_tmap_chunks(map, base, krows, cols, ld, 2 * BK, tile_cols / 64);
}

bool make_tmap_bf16_mn1(CUtensorMap* map, const void* base, uint64_t krows, uint64_t cols, uint64_t ld, uint32_t tile_cols) {
    return tile_cols % 64 == 0 && make_tmap_chunks(map, base, krows, cols, ld, BK, tile_cols / 64);
}

int tc_stage_blocks(int bn, int cm, int pair) { return (cm == 1 && !pair && bn <= 128) ? 2 : 1; }

bool make_tmap_out(CUtensorMap* map, void* base, bool fp32, uint64_t splits, uint64_t rows, uint64_t cols, uint64_t ld,
                   uint64_t split_ld) {
    EncodeTiledFn enc = get_encode();
    const uint64_t es = fp32 ? 4 : 2;
    if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15u) || (ld * es) % 16 || cols > ld || splits < 1 ||
        (splits > 1 && ((split_ld * es) % 16 || split_ld < rows * ld)))
        return false;
    cuuint64_t dims[3] = {cols, rows, splits};
    cuuint64_t strides[2] = {ld * es, (splits > 1 ? split_ld : rows * ld) * es};
    cuuint32_t box[3] = {fp32 ? 16u : 32u, 32u, 1u};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}


// Sets the dynamic shared-memory limit of every instantiation and measures how many clusters
// of each fit at once; called once per device before the first launch (and so before any
// stream capture).
cudaError_t tc_prepare() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    e = prepare_form<EPI_STORE, MAJ_K>(dev);
    e = e != cudaSuccess ? e : prepare_form<EPI_STORE, MAJ_MN>(dev);
    e = e != cudaSuccess ? e : prepare_form<EPI_BIAS_ELU, MAJ_K>(dev);
    e = e != cudaSuccess ? e : prepare_form<EPI_ELU_GRAD, MAJ_B_MN>(dev);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

int tc_cluster_fit(int bn, int epi, int cm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    const int bi = bn_index(bn), ci = cm_index(cm);
    if (bi < 0 || ci < 0 || epi < 0 || epi > 2) return 0;
    return g_fit[dev].clusters[bi][epi][ci];
}

int tc_ws_stages(int bn, int epi, int kblocks) {
    if (kblocks < 1) return 0;
    const bool g = epi == EPI_ELU_GRAD;
    switch (bn) {
        case 64: return g ? WsCfg<64, EPI_ELU_GRAD>::stages(kblocks) : WsCfg<64, EPI_BIAS_ELU>::stages(kblocks);
        case 128: return g ? WsCfg<128, EPI_ELU_GRAD>::stages(kblocks) : WsCfg<128, EPI_BIAS_ELU>::stages(kblocks);
        case 256: return g ? WsCfg<256, EPI_ELU_GRAD>::stages(kblocks) : WsCfg<256, EPI_BIAS_ELU>::stages(kblocks);
    }
    return 0;
}

int tc_smem_bytes(int bn, int epi) {
    switch (bn) {
        case 64: return epi == EPI_STORE ? TileCfg<64, EPI_STORE>::SMEM : TileCfg<64, EPI_BIAS_ELU>::SMEM;
        case 128: return epi == EPI_STORE ? TileCfg<128, EPI_STORE>::SMEM : TileCfg<128, EPI_BIAS_ELU>::SMEM;
        case 256: return epi == EPI_STORE ? TileCfg<256, EPI_STORE>::SMEM : TileCfg<256, EPI_BIAS_ELU>::SMEM;
    }
    return 0;
}

}  // namespace rl
