// Interface of the tcgen05 BF16 GEMM (see gemm_tc.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace rl {

enum { MAJ_K = 0, MAJ_MN = 1, MAJ_B_MN = 2 };

struct TcParams {
    CUtensorMap tmA[2];        // A operand per batch entry: [M][K] bf16, box 64 x 128 (see mn)
    CUtensorMap tmB[2];        // B operand per batch entry: [N][K] bf16, box 64 x (bn / cm)
    int M, N;                  // output rows / columns (N a multiple of bn)
    int kblocks;               // K / 64 (K zero-padded by TMA beyond the tensor)
    int kb_per_split, splits;  // split-K over blockIdx.z
    int batch;                 // 1 or 2 (actor, critic share one launch)
    int bn;                    // 64, 128 or 256
    int cm;                    // CTAs per cluster along M: 1, or 2 with pair (no copy is multicast)
    int pair;                  // with cm = 2: the pair runs one 256-row tile on the cta_group::2 MMA,
                               // each CTA loading half of B (B maps: box rows bn / 2); bn 128 / 256
    int mn;                    // operand forms: MAJ_K (A [M][K], B [N][K]), MAJ_MN (A^T [K][M],
                               // B^T [K][N], EPI_STORE), MAJ_B_MN (A [M][K], B^T [K][N],
                               // EPI_ELU_GRAD); MN-major operands use 64 x 64 boxes
    int epi;                   // EPI_STORE (fp32 split partials), EPI_BIAS_ELU, EPI_ELU_GRAD (bf16 out)
    CUtensorMap tmC[2];        // output per batch entry, [splits][M][N] (make_tmap_out): fp32 for
                               // EPI_STORE (split z at z), bf16 otherwise (one split)
    const float* bias[2];      // EPI_BIAS_ELU
    const void* hsrc[2];       // EPI_ELU_GRAD: bf16 activation [M][ldh] whose ELU derivative scales
    int ldh;                   // the product (row stride a multiple of 8)
    float* colsum[2];          // EPI_ELU_GRAD: per-row-tile column sums [4 M/128][N]
    int* status;               // device status word
    int ks;                    // K blocks per stage: 0 / 1, or 2 (cm 1, no pair, bn <= 128) with the
                               // operand maps of make_tmap_bf16_k2 (K-major) / make_tmap_bf16_mn2
    int max_ctas;              // persistent CTAs at most (0: as many as fit, one per SM)
    int mn3;                   // 1 (cm 1, no pair, ks 0 / 1): the MN-major operands are the 3D maps of
                               // make_tmap_bf16_mn1 (one copy per operand and stage instead of one
                               // per 64-wide box); 0: 64 x 64 box maps
    int ws;                    // 1: weight-stationary (cm 1, no pair, one split; forward or input
                               // gradient): each CTA keeps one (batch entry, column tile) B slice in
                               // shared memory and streams its row tiles' A through the ring, A by
                               // the two-K-block maps of make_tmap_bf16_k2, B by the maps of the
                               // single-CTA form (K-major box 64 x bn; MN-major make_tmap_bf16_mn1,
                               // mn3 = 1); the grid is a whole number of CTAs per group
    int sred;                  // split-K partials (EPI_STORE, MAJ_MN, cm 1): 0 writes every split's
                               // partial through tmC; 1..8 reduces them in clusters of sred CTAs
                               // holding consecutive splits of one tile (one CTA per tile and split),
                               // writing splits / sred partials to sr_out
    float* sr_out[2];          // per batch entry: partial g of element (m, n) at g sr_split_ld + m sr_ld + n
    long long sr_ld, sr_split_ld;
    int b_early;               // ws only: no kernel that may still run when this one starts writes B, so
                               // the B slice is fetched before the wait for the preceding kernel
};

cudaError_t launch_tc_gemm(const TcParams& p, cudaStream_t s);
bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows);
// two-K-block stage maps (cols a multiple of 64): K-major operand [rows][K], box 2 x (64 x box_rows);
// MN-major operand [K rows][cols], box 128 K rows x tile_cols (tile_cols / 64 chunks of 64)
bool make_tmap_bf16_k2(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows);
bool make_tmap_bf16_mn2(CUtensorMap* map, const void* base, uint64_t krows, uint64_t cols, uint64_t ld, uint32_t tile_cols);
// one-K-block stage map of an MN-major operand [K rows][cols] (cols a multiple of 64): box 64 K rows
// x tile_cols (tile_cols / 64 chunks of 64, at most 4)
bool make_tmap_bf16_mn1(CUtensorMap* map, const void* base, uint64_t krows, uint64_t cols, uint64_t ld, uint32_t tile_cols);
// K blocks per stage for a tile shape: 2 for single-CTA tiles of width <= 128, else 1
int tc_stage_blocks(int bn, int cm, int pair);
// output map [splits][rows][cols] (row stride ld elements, split stride split_ld elements), boxes
// of 32 rows x 64 bytes (fp32: 16 columns, bf16: 32) x 1, 64-byte swizzle
bool make_tmap_out(CUtensorMap* map, void* base, bool fp32, uint64_t splits, uint64_t rows, uint64_t cols, uint64_t ld,
                   uint64_t split_ld);
int tc_smem_bytes(int bn, int epi);
// ring stages of the weight-stationary form beside a resident B slice of kblocks K blocks (0 or
// less: the slice does not fit)
int tc_ws_stages(int bn, int epi, int kblocks);
int tc_cluster_fit(int bn, int epi, int cm);   // clusters resident at once (after tc_prepare)
cudaError_t tc_prepare();

}  // namespace rl
