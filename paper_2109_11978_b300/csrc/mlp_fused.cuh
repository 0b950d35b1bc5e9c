// Interface of the fused forward of the three hidden layers (see mlp_fused.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace rl {

// H_l = ELU(H_{l-1} W_l^T + b_l), l = 0, 1, 2, H_{-1} = X, for `nnets` networks that share X
// (actor and critic, or the critic alone), one CTA per (128-row tile, network).
struct MlpParams {
    CUtensorMap tmX;          // X [M][K0] bf16, box 64 x 128 (make_tmap_bf16), rows past M read as zeros
    CUtensorMap tmW[2][3];    // per network j: W_l [N_l][K_l] bf16, box 64 x 128
    CUtensorMap tmH[2][3];    // per network j: H_l [M][N_l] bf16, box 64 x 128 (TMA store targets; only
                              // tmH[j][2] when store_hidden is 0)
    const float* bias[2][3];  // per network j: b_l [N_l] fp32
    int M, K0, N0, N1, N2;    // rows; K0 = layer 0's input width; N_l = layer l's output width
    int nnets;                // 1 or 2 (grid y)
    int store_hidden;         // 1: H_0 and H_1 are written too (the update keeps them for the backward)
    int b_early;              // 1: no kernel that may still run when this one starts writes W or b, so
                              // the first weight blocks are fetched before the wait for it
    int* status;              // device status word (RL_ERR_TIMEOUT from a bounded wait)
};

// Widths the fused form takes: K0 a multiple of 64 in [64, 256], N0 a multiple of 128 in [128, 512],
// N1 and N2 multiples of 128 in [128, 256].
bool mlp_fwd_fits(int K0, int N0, int N1, int N2);
cudaError_t launch_mlp_fwd(const MlpParams& p, cudaStream_t s);
cudaError_t mlp_prepare();    // once per device before the first launch (and before any capture)

}  // namespace rl
