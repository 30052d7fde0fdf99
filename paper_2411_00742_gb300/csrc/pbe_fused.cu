// Fused path for one grid: a single persistent cooperative launch runs the
// whole solve.  Each block owns a fixed set of tiles; the two stages of every
// step are separated by a device-wide barrier.  After each barrier the block
// splits: warp 0 sums the per-block moment partials in a fixed order and
// advances the block's private copy of the scalar chain (solute balance,
// kinetics, CFL step - identical in every block), while the other warps
// already load the next stage's input tile and compute its face values,
// which do not depend on the kinetics.  Face quotients use the
// Newton-Raphson form (half_psi_fast).
//
// GB300 FP64 notes that shape this kernel: a warp-wide FP64 instruction
// occupies the SM's FP64 pipe for ~16 cycles whatever its active lanes, and
// a dependent FP64 operation takes ~65 cycles.  So (a) with one tile per
// block the moment weights of each thread's cells are computed once and
// kept in registers, (b) block reductions go through shared memory in two
// 16-wide levels instead of per-warp butterflies (3x fewer FP64 warp
// instructions), (c) the cross-block sum reads all partials with one load
// round and reduces every moment at once.
//
// Every wait is bounded: a barrier that does not complete within about one
// second sets PBE_ETIMEOUT and the kernel returns.
#include <type_traits>

#include "pbe_internal.h"
#include "pbe_tiles.cuh"

namespace pbe {

constexpr int kFNT = 256;     // threads per block (the reductions assume 256)
constexpr int kFT1 = 1024;    // 1-D tile
constexpr int kFTI = 16;      // 2-D tile rows
constexpr int kFTJ = 32;      // 2-D tile columns
constexpr long long kBarrierCycles = 2000000000LL;  // default wait limit: ~1 s at 2 GHz

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
// bar[0] counts arrivals and only grows: the k-th barrier completes when it
// reaches k * gridDim.x.  Thread 0 arrives with a release add (cumulative
// over the writes the block barrier ordered before it) and waits with
// acquire loads.  Returns false when the wait runs past `limit` cycles.
__device__ __forceinline__ unsigned int atom_add_release(unsigned int* p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ bool grid_barrier(unsigned int* bar, unsigned int& gen, int* fail_sh, long long limit)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = (gen + 1u) * gridDim.x;
        int ok = 1;
        const unsigned int arrived = atom_add_release(&bar[0], 1u) + 1u;
        if (arrived < target) {
            const long long t0 = clock64();
            unsigned int polls = 0;
            const unsigned int spin = limit > 0 ? 64u : 1u;
            while (ld_acquire(&bar[0]) < target) {
                if (++polls > spin) {
                    if (clock64() - t0 > limit) { ok = 0; break; }
                    __nanosleep(20);
                }
            }
        }
        gen += 1u;
        *fail_sh = !ok;
    }
    __syncthreads();
    return *fail_sh == 0;
}

// Block sum of one value (256 threads): warp butterflies, then thread 0 adds
// the eight warp sums as a balanced tree.  Result in *res (shared).
__device__ __forceinline__ void block_sum1(double v, double* wsum, double* res)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) *res = ((wsum[0] + wsum[1]) + (wsum[2] + wsum[3])) + ((wsum[4] + wsum[5]) + (wsum[6] + wsum[7]));
    __syncthreads();
}

// Cross-block sums of all NV slots by one warp: lane l < 3*NV sums slot
// l % NV over the blocks b = l / NV (mod 3) as balanced trees of 16, then
// the three lanes of each slot are added in a fixed order; lanes 0..NV-1
// write the totals to out[].
template <int NV>
__device__ __forceinline__ void warp_sum_partials_all(const double* part, int G, double* out)
{
    const int lane = threadIdx.x & 31;
    const int v = lane % NV, ph = lane / NV;
    double acc = 0.0;
    if (ph < 3) {
        for (int base = ph; base < G; base += 3 * 16) {
            double a[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int b = base + 3 * q;
                a[q] = b < G ? __ldcg(part + (size_t)b * kMaxMom + v) : 0.0;
            }
#pragma unroll
            for (int w = 8; w > 0; w >>= 1)
#pragma unroll
                for (int q = 0; q < w; ++q) a[q] += a[q + w];
            acc += a[0];
        }
    }
    const double a1 = __shfl_sync(0xffffffffu, acc, (lane + NV) & 31);
    const double a2 = __shfl_sync(0xffffffffu, acc, (lane + 2 * NV) & 31);
    if (lane < NV) out[lane] = (acc + a1) + a2;
}

// Deterministic block sum of NV values per thread through shared memory:
// 16 threads per value each sum 16 rows (balanced tree), then one thread per
// value sums the 16 results.  Result in res[0..NV) (shared).  256 threads.
template <int NV>
__device__ __forceinline__ void block_sum_smem(const double (&v)[NV], double* red, double* red2, double* res)
{
    constexpr int S = NV + 1;
#pragma unroll
    for (int k = 0; k < NV; ++k) red[threadIdx.x * S + k] = v[k];
    __syncthreads();
    const int vv = threadIdx.x & 15, ch = threadIdx.x >> 4;
    if (vv < NV) {
        double a[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) a[r] = red[(ch * 16 + r) * S + vv];
#pragma unroll
        for (int w = 8; w > 0; w >>= 1)
#pragma unroll
            for (int r = 0; r < w; ++r) a[r] += a[r + w];
        red2[ch * 16 + vv] = a[0];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double a[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) a[r] = red2[r * 16 + threadIdx.x];
#pragma unroll
        for (int w = 8; w > 0; w >>= 1)
#pragma unroll
            for (int r = 0; r < w; ++r) a[r] += a[r + w];
        res[threadIdx.x] = a[0];
    }
    __syncthreads();
}

// Cross-block sums of NV moment slots (slot[k]) by one warp in a fixed
// order: lanes read 4 partials per round, tree-sum them, then a butterfly;
// every lane ends with the totals.
template <int NV>
__device__ __forceinline__ void warp_sum_partials(const double* part, int G, const int (&slot)[NV], double (&tot)[NV])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = 0.0;
    for (int base = 0; base < G; base += 128) {
        double v[NV][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = base + lane + 32 * q;
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k][q] = b < G ? __ldcg(part + (size_t)b * kMaxMom + slot[k]) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] += (v[k][0] + v[k][2]) + (v[k][1] + v[k][3]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] += __shfl_xor_sync(0xffffffffu, tot[k], o);
}

// In the window after each barrier warp 0 runs the scalar chain, warps 1-6
// compute the next stage's faces (enough to keep the FP64 pipe busy while
// leaving issue slots to warp 0's dependent chain) and warp 7 reduces the
// deferred output moments (warp 7).
constexpr int kFaceWarps = 6;
struct GroupSync {  // named barrier over the face warps 1..kFaceWarps
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync 1, %0;" ::"r"(32 * kFaceWarps) : "memory"); }
};
struct MomSync {    // named barrier over warps kFaceWarps+1..7
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync 2, %0;" ::"r"(kFNT - 32 * (kFaceWarps + 1)) : "memory"); }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

template <int NDIM>
struct FusedSmem;
template <>
struct FusedSmem<1> {
    double tile[kFT1 + 3];
    double h[kFT1 + 1];
};
template <>
struct FusedSmem<2> {
    Tile2DSmem<kFTI, kFTJ> t;
};

template <int NDIM>
struct TileShape;
template <>
struct TileShape<1> {
    static constexpr int CELLS = kFT1;
};
template <>
struct TileShape<2> {
    static constexpr int CELLS = kFTI * kFTJ;
};

template <int NDIM>
__device__ __forceinline__ void tile_origin(int t, int tiles_x, int& i0, int& j0)
{
    if (NDIM == 1) { i0 = t * kFT1; j0 = 0; }
    else { i0 = (t / tiles_x) * kFTI; j0 = (t % tiles_x) * kFTJ; }
}

// local cell q of this thread in a tile -> (i, j)
template <int NDIM>
__device__ __forceinline__ void cell_of(int k, int i0, int j0, int& i, int& j, int& r, int& c)
{
    if (NDIM == 1) { r = k; c = 0; i = i0 + k; j = 0; }
    else { r = k / kFTJ; c = k - r * kFTJ; i = i0 + r; j = j0 + c; }
}

// moment weights of cell (i, j): x^k dL (1-D), x1^p x2^q dA (2-D, row order)
template <int NDIM>
__device__ __forceinline__ void moment_weights(int i, int j, const Geom& g, double* w)
{
    if (NDIM == 1) {
        const double x = (i + 0.5) * g.d1;
        w[0] = g.d1; w[1] = x * w[0]; w[2] = x * w[1]; w[3] = x * w[2];
    } else {
        const double x1 = (i + 0.5) * g.d1, x2 = (j + 0.5) * g.d2;
        const double a = g.d1 * g.d2;
        const double a1 = x1 * a, a2 = x2 * a;
        w[0] = a; w[1] = a1; w[2] = a2;
        w[3] = x1 * a1; w[4] = x1 * a2; w[5] = x2 * a2;
        w[6] = x1 * x1 * a1; w[7] = x1 * x1 * a2; w[8] = x1 * x2 * a2; w[9] = x2 * x2 * a2;
    }
}

template <int NDIM, class Sync>
__device__ __forceinline__ void fused_faces(const double* in, int t, int tiles_x, const Geom& g, FusedSmem<NDIM>& sm,
                                            int tid, int nthr, Sync sync)
{
    int i0, j0;
    tile_origin<NDIM>(t, tiles_x, i0, j0);
    if constexpr (NDIM == 1) faces1d<true, true, kFT1>(in, i0, g, sm.tile, sm.h, tid, nthr, sync);
    else faces2d<true, true, kFTI, kFTJ>(in, i0, j0, g, sm.t, tid, nthr, sync);
}

// update of cell local index k of tile (i0, j0) from the faces in shared memory
template <int STAGE, int NDIM>
__device__ __forceinline__ double cell_update(const double* old, double* out, int k, int i0, int j0, const Geom& g,
                                              const StageCoef& sc, const FusedSmem<NDIM>& sm, bool& valid, int& i,
                                              int& j)
{
    int r, c;
    cell_of<NDIM>(k, i0, j0, i, j, r, c);
    valid = (NDIM == 1) ? (i < g.N1) : (i < g.N1 && j < g.N2);
    if (!valid) return 0.0;
    double v;
    size_t gidx;
    if constexpr (NDIM == 1) {
        v = sm.tile[r + 2] + sc.c1 * (sm.h[r] - sm.h[r + 1]);
        gidx = i;
        if (i == 0) v += sc.src;
    } else {
        constexpr int W = kFTJ + 3;
        const auto& s = sm.t;
        v = s.tile[(r + 2) * W + c + 2] + sc.c1 * (s.h1[r * kFTJ + c] - s.h1[(r + 1) * kFTJ + c]) +
            sc.c2 * (s.h2[r * (kFTJ + 1) + c] - s.h2[r * (kFTJ + 1) + c + 1]);
        gidx = (size_t)i * g.N2 + j;
        if (i == 0 && j == 0) v += sc.src;
    }
    if (STAGE == 2) v = 0.5 * old[gidx] + 0.5 * v;
    out[gidx] = v;
    return v;
}

template <int NDIM, bool ONE_TILE>
__global__ void __launch_bounds__(kFNT, 1) k_fused(double* n, double* n1, Scal* S, Kin K, Geom g, double* part,
                                                   const double* t_out, double* rows, unsigned int* bar, int ntiles,
                                                   int tiles_x, long long wait_limit, double* rowpart)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    constexpr int CPT = TileShape<NDIM>::CELLS / kFNT;   // cells per thread per tile
    __shared__ Scal s;
    __shared__ StageCoef scs;   // coefficients of the coming stage (written by thread 0)
    __shared__ double red[kFNT * (NM + 1)];
    __shared__ double red2[256];
    __shared__ double res[NM];
    __shared__ double msum[NM];
    __shared__ int fail;
    __shared__ FusedSmem<NDIM> sm;
    if (threadIdx.x == 0) {
        s = *S;
        s.row_first = s.out_idx;   // rows before this index came from the prologue
        scs = stage_coef_fast<1>(s, g);
    }
    __syncthreads();
    if (s.done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) S->row_first = s.row_first;
        return;
    }
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5;
    double* part1 = part;                        // stage-1 partials [G][kMaxMom]
    double* part2 = part + (size_t)G * kMaxMom;  // stage-2 partials
    double* my_rows = blockIdx.x == 0 ? rows : nullptr;
    unsigned int gen = 0;

    // moment weights of this thread's cells (one tile per block: fixed for the whole solve)
    double wgt[ONE_TILE ? CPT : 1][ONE_TILE ? NM : 1];
    if constexpr (ONE_TILE) {
        int i0, j0;
        tile_origin<NDIM>(blockIdx.x, tiles_x, i0, j0);
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            int i, j, r, c;
            cell_of<NDIM>(threadIdx.x + q * kFNT, i0, j0, i, j, r, c);
            moment_weights<NDIM>(i, j, g, wgt[q]);
        }
    }

    fused_faces<NDIM>(n, blockIdx.x, tiles_x, g, sm, threadIdx.x, kFNT, BlockSync());
    __syncthreads();
    for (;;) {
#pragma unroll 1
        for (int stage = 1; stage <= 2; ++stage) {
            const StageCoef sc = scs;
            const double* in = stage == 1 ? n : n1;
            double* out = stage == 1 ? n1 : n;
            double m[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) m[k] = 0.0;
            for (int t = blockIdx.x; t < ntiles; t += G) {
                if (t != (int)blockIdx.x) {
                    fused_faces<NDIM>(in, t, tiles_x, g, sm, threadIdx.x, kFNT, BlockSync());
                    __syncthreads();
                }
                int i0, j0;
                tile_origin<NDIM>(t, tiles_x, i0, j0);
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    bool valid;
                    int i, j;
                    const double v = stage == 1 ? cell_update<1, NDIM>(n, out, threadIdx.x + q * kFNT, i0, j0, g, sc, sm, valid, i, j)
                                                : cell_update<2, NDIM>(n, out, threadIdx.x + q * kFNT, i0, j0, g, sc, sm, valid, i, j);
                    if (!valid) continue;
                    double wl[NM];
                    if constexpr (ONE_TILE) {
#pragma unroll
                        for (int k = 0; k < NM; ++k) wl[k] = wgt[q][k];
                    } else {
                        moment_weights<NDIM>(i, j, g, wl);
                    }
                    if (sc.moms) {
#pragma unroll
                        for (int k = 0; k < NM; ++k) m[k] += wl[k] * v;
                    } else {
                        m[VIDX] += wl[VIDX] * v;
                    }
                }
                __syncthreads();
            }
            double* pp = stage == 1 ? part1 : part2;
            const int row_here = s.out_idx;
            // only the volume moment is on the critical path; on output steps
            // the per-thread moments wait in shared memory and are reduced in
            // the overlap window, the row completed after the solve
            if (sc.moms) {
#pragma unroll
                for (int k = 0; k < NM; ++k) red[threadIdx.x * (NM + 1) + k] = m[k];
            }
            block_sum1(m[VIDX], red2, res);
            if (threadIdx.x == 0) pp[(size_t)blockIdx.x * kMaxMom + VIDX] = res[0];
            if (!grid_barrier(bar, gen, &fail, wait_limit)) break;
            if (warp == 0) {
                const int slots[1] = {VIDX};
                double tot[1];
                warp_sum_partials<1>(pp, G, slots, tot);
                if (threadIdx.x == 0) msum[VIDX] = tot[0];
                __syncwarp();
                if (stage == 1) finish_stage1_warp(&s, K, msum[VIDX]);
                else finish_stage2_warp(&s, K, g, t_out, my_rows, msum, NM, VIDX);
                // the next stage's coefficients, once per block (the divisions of
                // stage_coef in every thread cost the FP64 pipe ~4k cycles a stage)
                if (threadIdx.x == 0) scs = stage == 1 ? stage_coef_fast<2>(s, g) : stage_coef_fast<1>(s, g);
            } else if (warp <= kFaceWarps) {
                // faces of the next stage's input for this block's first tile
                fused_faces<NDIM>(stage == 1 ? n1 : n, blockIdx.x, tiles_x, g, sm, threadIdx.x - 32, 32 * kFaceWarps,
                                  GroupSync());
            } else if (sc.moms) {
                // two-level sum of the block's moments: 16 threads per moment, then one
                constexpr int NT2 = kFNT - 32 * (kFaceWarps + 1);
                const int t0 = threadIdx.x - 32 * (kFaceWarps + 1);
                for (int t = t0; t < 16 * NM; t += NT2) {
                    const int v = t >> 4, ch = t & 15;
                    double a[16];
#pragma unroll
                    for (int r = 0; r < 16; ++r) a[r] = red[(ch * 16 + r) * (NM + 1) + v];
#pragma unroll
                    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
                        for (int r = 0; r < w; ++r) a[r] += a[r + w];
                    red2[256 - 16 * NM + v * 16 + ch] = a[0];
                }
                MomSync()();
                if (t0 < NM) {
                    double a[16];
#pragma unroll
                    for (int r = 0; r < 16; ++r) a[r] = red2[256 - 16 * NM + t0 * 16 + r];
#pragma unroll
                    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
                        for (int r = 0; r < w; ++r) a[r] += a[r + w];
                    rowpart[((size_t)row_here * G + blockIdx.x) * NM + t0] = a[0];
                }
            }
            __syncthreads();
            if (s.done) break;
        }
        if (s.done || fail) break;
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

// Moments of the rows the fused solve emitted: sums of the per-block partials
// in block order (one block per row, one thread per moment).
template <int NDIM>
__global__ void k_fused_rows(const double* rowpart, int G, const Scal* S, double* rows)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    const int r = S->row_first + blockIdx.x;
    if (r >= S->out_idx || threadIdx.x >= NM) return;
    double acc = 0.0;
    for (int b = 0; b < G; ++b) acc += rowpart[((size_t)r * G + b) * NM + threadIdx.x];
    rows[(size_t)r * (NM + 2) + 1 + threadIdx.x] = acc;
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
    int tiles_x;
    const int ntiles = fused_tiles(g->geo, &tiles_x);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) return e;
    const bool one = g->geo.ndim == 1 ? true : true;
    const void* fn_multi = g->geo.ndim == 1 ? (const void*)k_fused<1, false> : (const void*)k_fused<2, false>;
    const void* fn_one = g->geo.ndim == 1 ? (const void*)k_fused<1, true> : (const void*)k_fused<2, true>;
    (void)one;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn_one, kFNT, 0);
    if (e != cudaSuccess) return e;
    int G = ntiles;
    if (G > occ * sms) G = occ * sms;
    if (2 * G > g->max_blocks) G = g->max_blocks / 2;
    if (G < 1) G = 1;
    const void* fn = (G >= ntiles) ? fn_one : fn_multi;
    if (fn == fn_multi) {
        int occ2 = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, fn_multi, kFNT, 0);
        if (e != cudaSuccess) return e;
        if (G > occ2 * sms) G = occ2 * sms;
    }
    e = cudaMemsetAsync(g->d_bar, 0, 2 * sizeof(unsigned int), g->stream);
    if (e != cudaSuccess) return e;
    long long wait_limit = g->wait_cycles > 0 ? g->wait_cycles : (g->wait_cycles == 0 ? 0 : kBarrierCycles);
    void* args[] = {&g->d_n, &g->d_n1, &g->d_S, &g->kin, &g->geo, &g->d_part, &g->d_tout, &g->d_rows,
                    &g->d_bar, (void*)&ntiles, &tiles_x, &wait_limit, &g->d_rowpart};
    e = cudaLaunchCooperativeKernel(fn, G, kFNT, args, 0, g->stream);
    if (e != cudaSuccess) return e;
    const int nrows = n_out > 0 ? n_out : 1;
    if (g->geo.ndim == 1) k_fused_rows<1><<<nrows, 32, 0, g->stream>>>(g->d_rowpart, G, g->d_S, g->d_rows);
    else k_fused_rows<2><<<nrows, 32, 0, g->stream>>>(g->d_rowpart, G, g->d_S, g->d_rows);
    return cudaGetLastError();
}

}  // namespace pbe
