// Procedural terrain family (Sec. 3.1, Fig. 2): the heightfield of the curriculum grid, tile rows
// = levels (difficulty grows with the row), tile columns = terrain kinds.  Five types: flat,
// sloped, randomly rough, discrete obstacles, stairs; slopes and stairs as pyramids (up) and pits
// (down) so that robots both climb and descend them.  With the level's difficulty d in [0, 1]:
// slope inclination 25 deg x d, stair and obstacle step height 0.05 + 0.15 d m; stairs 0.3 m wide,
// rough terrain with 0.1 m of variation, obstacles on 1 m blocks; a flat 2 m x 2 m platform at the
// tile centre where robots spawn.  One thread per grid point; random heights from the
// counter-based generator keyed by (seed, terrain stream, level, column), so the field depends on
// the seed only.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

constexpr float SLOPE_MAX_RAD = 0.43633231299858238f;   // 25 deg
constexpr float STEP_MIN = 0.05f, STEP_RANGE = 0.15f;  // 0.05 m -> 0.20 m
constexpr float ROUGH_RANGE = 0.1f;

__global__ void __launch_bounds__(256) terrain_kernel(TerrainParams p, float* __restrict__ hf) {
    pdl_wait();
    pdl_trigger();
    const long long ny = (long long)p.cols * p.c, n = (long long)p.levels * p.c * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i / ny), y = (int)(i - (long long)x * ny);
        const int lvl = x / p.c, k = y / p.c, a = x - lvl * p.c, b = y - k * p.c;
        const float d = p.levels > 1 ? (float)lvl / (float)(p.levels - 1) : 0.f;
        const float step = STEP_MIN + STEP_RANGE * d;
        // cells to the tile border, capped at the platform's edge
        const int e = min(min(min(a, b), min(p.c - a, p.c - b)), p.c / 2 - p.P);
        float h = 0.f;
        switch (k % 7) {
            case 1:   // slope pyramid
            case 2: {  // slope pit
                const float s = tanf(SLOPE_MAX_RAD * d) * (float)e * p.res;
                h = (k % 7) == 1 ? s : -s;
                break;
            }
            case 3: {  // randomly rough
                const uint64_t key = rng_key(p.seed, kStreamTerrain, (uint64_t)lvl, (uint64_t)k, 0);
                h = ROUGH_RANGE * (uniform01(hi32(rng_word(key, (uint32_t)(a * p.c + b)))) - 0.5f);
                break;
            }
            case 4: {  // discrete obstacles on blocks, the platform's blocks flat
                const int nb = p.c / p.B, ba = a / p.B, bb = b / p.B;
                if (abs(2 * ba + 1 - nb) <= 1 && abs(2 * bb + 1 - nb) <= 1) break;
                const uint64_t key = rng_key(p.seed, kStreamTerrain, (uint64_t)lvl, (uint64_t)k, 1);
                h = step * uniform_pm1(hi32(rng_word(key, (uint32_t)(ba * nb + bb))));
                break;
            }
            case 5:   // stairs pyramid
            case 6: {  // stairs pit
                const float s = step * (float)(e / p.W);
                h = (k % 7) == 5 ? s : -s;
                break;
            }
            default:  // flat
                break;
        }
        hf[i] = h;
    }
}

}  // namespace

cudaError_t launch_terrain(const TerrainParams& p, float* hf, cudaStream_t s) {
    const long long n = (long long)p.levels * p.c * p.cols * p.c;
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((n + 255) / 256, 148 * 16);
    cudaError_t e = launch_pdl(terrain_kernel, dim3(grid), dim3(256), 0, s, p, hf);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rl
