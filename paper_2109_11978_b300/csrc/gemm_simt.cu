// FP32 CUDA-core GEMM for the plain FP32 form of the actor/critic MLPs (forward, input
// gradient and weight gradient), with the bias + ELU, ELU-derivative and split-K epilogues
// fused.  This is the FP32 baseline the BF16 tensor-core form is compared against.
//
// Tile 128 x 64 x 16, 256 threads, 8 x 4 outputs per thread, double-buffered shared memory.
// A and B may each be "k-major" (k contiguous) or "m/n-major"; the loads are float4 along the
// contiguous dimension either way, so every layout the MLP needs is read coalesced:
//   forward  Y = X W^T:   A = X [M][K],        B = W [N][K]
//   input    dX = dY W:   A = dY [M][N_l],     B = W [N_l][K_l]   (b_t)
//   weight   dW = dY^T X: A = dY [rows][N_l]   (a_t), B = X [rows][K_l] (b_t), split over rows
#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

constexpr int BM = 128, BN = 64, BK = 16, NT = 256;

template <int EPI, bool AT, bool BT>
__global__ void __launch_bounds__(NT) gemm_f32_kernel(int M, int N, int K, int lda, int ldb, int ldc, int ldh,
                                                      int splits, int kchunk, GemmBatch g) {
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int bz = blockIdx.z, b = bz / splits, sp = bz % splits;
    const float* __restrict__ A = g.A[b];
    const float* __restrict__ B = g.B[b];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kbeg = sp * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    float4 ra[2], rb;
    auto load_regs = [&](int k0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int f = tid + i * NT;
            if (!AT) {
                const int m = f >> 2, kq = (f & 3) * 4;
                ra[i] = (m0 + m < M) ? __ldg(reinterpret_cast<const float4*>(A + (size_t)(m0 + m) * lda + k0 + kq))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const int k = f >> 5, mq = (f & 31) * 4;
                ra[i] = (m0 + mq < M) ? __ldg(reinterpret_cast<const float4*>(A + (size_t)(k0 + k) * lda + m0 + mq))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (!BT) {
            const int n = tid >> 2, kq = (tid & 3) * 4;
            rb = __ldg(reinterpret_cast<const float4*>(B + (size_t)(n0 + n) * ldb + k0 + kq));
        } else {
            const int k = tid >> 4, nq = (tid & 15) * 4;
            rb = __ldg(reinterpret_cast<const float4*>(B + (size_t)(k0 + k) * ldb + n0 + nq));
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int f = tid + i * NT;
            if (!AT) {
                const int m = f >> 2, kq = (f & 3) * 4;
                As[buf][kq + 0][m] = ra[i].x; As[buf][kq + 1][m] = ra[i].y;
                As[buf][kq + 2][m] = ra[i].z; As[buf][kq + 3][m] = ra[i].w;
            } else {
                const int k = f >> 5, mq = (f & 31) * 4;
                *reinterpret_cast<float4*>(&As[buf][k][mq]) = ra[i];
            }
        }
        if (!BT) {
            const int n = tid >> 2, kq = (tid & 3) * 4;
            Bs[buf][kq + 0][n] = rb.x; Bs[buf][kq + 1][n] = rb.y; Bs[buf][kq + 2][n] = rb.z; Bs[buf][kq + 3][n] = rb.w;
        } else {
            const int k = tid >> 4, nq = (tid & 15) * 4;
            *reinterpret_cast<float4*>(&Bs[buf][k][nq]) = rb;
        }
    };

    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    int buf = 0;
    if (kbeg < kend) {
        load_regs(kbeg);
        store_smem(0);
    }
    __syncthreads();
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        const bool more = k0 + BK < kend;
        if (more) load_regs(k0 + BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8 + 4]);
            const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bw[j], acc[i][j]);
        }
        if (more) store_smem(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }

    float* __restrict__ C = g.C[b];
    const int c0 = n0 + tx * 4;
    if (EPI == EPI_STORE) C += (size_t)sp * g.split_stride;
    float4 bias4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (EPI == EPI_BIAS_ELU) bias4 = __ldg(reinterpret_cast<const float4*>(g.bias[b] + c0));
    float cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = m0 + ty * 8 + i;
        if (r >= M) break;
        float4 o = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        if (EPI == EPI_BIAS_ELU) {
            o.x = elu(o.x + bias4.x); o.y = elu(o.y + bias4.y); o.z = elu(o.z + bias4.z); o.w = elu(o.w + bias4.w);
        } else if (EPI == EPI_ELU_GRAD) {
            const float4 h = __ldg(reinterpret_cast<const float4*>(g.H[b] + (size_t)r * ldh + c0));
            o.x *= elu_grad_y(h.x); o.y *= elu_grad_y(h.y); o.z *= elu_grad_y(h.z); o.w *= elu_grad_y(h.w);
            cs[0] += o.x; cs[1] += o.y; cs[2] += o.z; cs[3] += o.w;
        }
        *reinterpret_cast<float4*>(C + (size_t)r * ldc + c0) = o;
    }
    if (EPI == EPI_ELU_GRAD && g.colsum[b]) {
        // column sums of this row tile (the bias gradient of the layer below)
        float (*red)[BN] = reinterpret_cast<float (*)[BN]>(&As[0][0][0]);   // 16 x 64 floats, reuse
#pragma unroll
        for (int j = 0; j < 4; ++j) red[ty][tx * 4 + j] = cs[j];
        __syncthreads();
        if (tid < BN) {
            float s = 0.f;
#pragma unroll
            for (int y = 0; y < 16; ++y) s += red[y][tid];
            g.colsum[b][(size_t)blockIdx.x * N + n0 + tid] = s;
        }
    }
}

template <int EPI>
cudaError_t dispatch(bool a_t, bool b_t, dim3 grid, int M, int N, int K, int lda, int ldb, int ldc, int ldh,
                     int splits, int kchunk, const GemmBatch& g, cudaStream_t s) {
    if (!a_t && !b_t) { cudaError_t e = launch_pdl(gemm_f32_kernel<EPI, false, false>, grid, dim3(NT), 0, s, M, N, K, lda, ldb, ldc, ldh, splits, kchunk, g); if (e != cudaSuccess) return e; }
    else if (!a_t && b_t) { cudaError_t e = launch_pdl(gemm_f32_kernel<EPI, false, true>, grid, dim3(NT), 0, s, M, N, K, lda, ldb, ldc, ldh, splits, kchunk, g); if (e != cudaSuccess) return e; }
    else if (a_t && !b_t) { cudaError_t e = launch_pdl(gemm_f32_kernel<EPI, true, false>, grid, dim3(NT), 0, s, M, N, K, lda, ldb, ldc, ldh, splits, kchunk, g); if (e != cudaSuccess) return e; }
    else { cudaError_t e = launch_pdl(gemm_f32_kernel<EPI, true, true>, grid, dim3(NT), 0, s, M, N, K, lda, ldb, ldc, ldh, splits, kchunk, g); if (e != cudaSuccess) return e; }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_f32(int epi, bool a_t, bool b_t, int M, int N, int K, int lda, int ldb, int ldc, int ldh,
                            int batch, int splits, int kchunk, const GemmBatch& g, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (N % BN || K % BK || kchunk % BK || (a_t && M % 4)) return cudaErrorInvalidValue;
    dim3 grid((M + BM - 1) / BM, N / BN, batch * splits);
    switch (epi) {
        case EPI_STORE: return dispatch<EPI_STORE>(a_t, b_t, grid, M, N, K, lda, ldb, ldc, ldh, splits, kchunk, g, s);
        case EPI_BIAS_ELU: return dispatch<EPI_BIAS_ELU>(a_t, b_t, grid, M, N, K, lda, ldb, ldc, ldh, splits, kchunk, g, s);
        case EPI_ELU_GRAD: return dispatch<EPI_ELU_GRAD>(a_t, b_t, grid, M, N, K, lda, ldb, ldc, ldh, splits, kchunk, g, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rl
