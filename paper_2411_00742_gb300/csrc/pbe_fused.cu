// Fused path for one grid: a single persistent cooperative launch runs the
// whole solve.  Each block owns a fixed set of tiles; the two stages of every
// step are separated by a device-wide barrier, after which every block
// reduces the per-block moment partials in the same fixed order and advances
// an identical private copy of the scalar chain (kinetics, CFL step, solute
// balance), so the only device-wide traffic per stage is one barrier and the
// partials.  Face quotients use the Newton-Raphson form (half_psi_fast).
//
// Every wait is bounded: a barrier that does not complete within about one
// second sets PBE_ETIMEOUT and the kernel returns.
#include "pbe_internal.h"
#include "pbe_tiles.cuh"

#include <type_traits>

namespace pbe {

constexpr int kFNT = 256;     // threads per block
constexpr int kFT1 = 1024;    // 1-D tile
constexpr int kFTI = 8;       // 2-D tile rows
constexpr int kFTJ = 32;      // 2-D tile columns
constexpr long long kBarrierCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Device-wide barrier over gridDim.x co-resident blocks (cooperative launch).
// bar[0] counts arrivals, bar[1] is the generation.  Returns false on timeout.
__device__ bool grid_barrier(unsigned int* bar, unsigned int& gen, int* fail_sh)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = gen + 1u;
        int ok = 1;
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar[0], 1u);
        if (arrived == gridDim.x - 1u) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            st_release(&bar[1], target);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(&bar[1]) != target) {
                if (clock64() - t0 > kBarrierCycles) { ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        gen = target;
        *fail_sh = !ok;
    }
    __syncthreads();
    return *fail_sh == 0;
}

template <int NV>
__device__ __forceinline__ void reduce_slot(const double* part, int nblocks, double (&v)[NV], double* sh)
{
    reduce_partials<kFNT, NV>(part, nblocks, v, sh);
}

template <int NDIM>
__global__ void __launch_bounds__(kFNT) k_fused(double* n, double* n1, Scal* S, Kin K, Geom g, double* part,
                                                const double* t_out, double* rows, unsigned int* bar, int ntiles,
                                                int tiles_x)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    __shared__ Scal s;
    __shared__ double sh[kFNT / 32 * NM];
    __shared__ int fail;
    __shared__ typename std::conditional<NDIM == 1, double[2 * kFT1 + 4], Tile2DSmem<kFTI, kFTJ>>::type smem;
    if (threadIdx.x == 0) s = *S;
    __syncthreads();
    if (s.done) return;
    unsigned int gen = 0;
    const int G = gridDim.x;
    double* part1 = part;                          // stage-1 partials [G][kMaxMom]
    double* part2 = part + (size_t)G * kMaxMom;    // stage-2 partials
    double* my_rows = blockIdx.x == 0 ? rows : nullptr;
    for (;;) {
        // ---- stage 1: n1 = n + dt L(n) ----
        {
            const StageCoef sc = stage_coef<1>(s, g);
            double m[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) m[k] = 0.0;
            for (int t = blockIdx.x; t < ntiles; t += G) {
                if constexpr (NDIM == 1) {
                    double* sm = reinterpret_cast<double*>(&smem);
                    tile1d<1, true, true, kFT1, kFNT>(n, n, n1, t * kFT1, g, sc, *reinterpret_cast<double(*)[4]>(m),
                                                      sm, sm + kFT1 + 3);
                } else {
                    auto& ts = *reinterpret_cast<Tile2DSmem<kFTI, kFTJ>*>(&smem);
                    tile2d<1, true, true, kFTI, kFTJ, kFNT>(n, n, n1, (t / tiles_x) * kFTI, (t % tiles_x) * kFTJ, g, sc,
                                                           *reinterpret_cast<double(*)[10]>(m), ts);
                }
            }
            double v[1] = {m[VIDX]};
            block_sum<kFNT, 1>(v, sh);
            if (threadIdx.x == 0) part1[(size_t)blockIdx.x * kMaxMom + VIDX] = v[0];
            if (!grid_barrier(bar, gen, &fail)) break;
            // every block sums the volume partials in the same order
            double r[1] = {0.0};
            for (int b = threadIdx.x; b < G; b += kFNT) r[0] += __ldcg(part1 + (size_t)b * kMaxMom + VIDX);
            block_sum<kFNT, 1>(r, sh);
            if (threadIdx.x == 0) finish_stage1(&s, K, r[0]);
            __syncthreads();
            if (s.done) break;
        }
        // ---- stage 2: n = n/2 + (n1 + dt L(n1))/2 ----
        {
            const StageCoef sc = stage_coef<2>(s, g);
            double m[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) m[k] = 0.0;
            for (int t = blockIdx.x; t < ntiles; t += G) {
                if constexpr (NDIM == 1) {
                    double* sm = reinterpret_cast<double*>(&smem);
                    tile1d<2, true, true, kFT1, kFNT>(n1, n, n, t * kFT1, g, sc, *reinterpret_cast<double(*)[4]>(m),
                                                      sm, sm + kFT1 + 3);
                } else {
                    auto& ts = *reinterpret_cast<Tile2DSmem<kFTI, kFTJ>*>(&smem);
                    tile2d<2, true, true, kFTI, kFTJ, kFNT>(n1, n, n, (t / tiles_x) * kFTI, (t % tiles_x) * kFTJ, g, sc,
                                                           *reinterpret_cast<double(*)[10]>(m), ts);
                }
            }
            block_sum<kFNT, NM>(m, sh);
            if (threadIdx.x == 0)
                for (int k = 0; k < NM; ++k) part2[(size_t)blockIdx.x * kMaxMom + k] = m[k];
            if (!grid_barrier(bar, gen, &fail)) break;
            for (int k = 0; k < NM; ++k) m[k] = 0.0;
            if (sc.moms) {
                reduce_slot<NM>(part2, G, m, sh);
            } else {
                double r[1] = {0.0};
                for (int b = threadIdx.x; b < G; b += kFNT) r[0] += __ldcg(part2 + (size_t)b * kMaxMom + VIDX);
                block_sum<kFNT, 1>(r, sh);
                m[VIDX] = r[0];
            }
            if (threadIdx.x == 0) finish_stage2(&s, K, g, t_out, my_rows, m, NM, VIDX);
            __syncthreads();
            if (s.done) break;
        }
    }
    if (threadIdx.x == 0 && fail) {
        S->status = PBE_ETIMEOUT;
        S->done = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !fail) {
        s.counter = 0u;
        *S = s;
    }
}

static int fused_tiles(const Geom& g, int* tiles_x)
{
    if (g.ndim == 1) {
        *tiles_x = 1;
        return (g.N1 + kFT1 - 1) / kFT1;
    }
    *tiles_x = (g.N2 + kFTJ - 1) / kFTJ;
    return *tiles_x * ((g.N1 + kFTI - 1) / kFTI);
}

bool fused_supported(const pbe_grid* g) { return g->d_bar != nullptr; }

cudaError_t launch_fused_solve(pbe_grid* g, int n_out)
{
    (void)n_out;
    int tiles_x;
    const int ntiles = fused_tiles(g->geo, &tiles_x);
    static thread_local int occ_cache[2] = {0, 0};
    int& occ = occ_cache[g->geo.ndim - 1];
    const void* fn = g->geo.ndim == 1 ? (const void*)k_fused<1> : (const void*)k_fused<2>;
    if (occ == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kFNT, 0);
        if (e != cudaSuccess) return e;
    }
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) return e;
    int G = ntiles;
    if (G > occ * sms) G = occ * sms;
    if (2 * G > g->max_blocks) G = g->max_blocks / 2;
    if (G < 1) G = 1;
    e = cudaMemsetAsync(g->d_bar, 0, 2 * sizeof(unsigned int), g->stream);
    if (e != cudaSuccess) return e;
    void* args[] = {&g->d_n, &g->d_n1, &g->d_S, &g->kin, &g->geo, &g->d_part, &g->d_tout, &g->d_rows,
                    &g->d_bar, (void*)&ntiles, &tiles_x};
    return cudaLaunchCooperativeKernel(fn, G, kFNT, args, 0, g->stream);
}

}  // namespace pbe
