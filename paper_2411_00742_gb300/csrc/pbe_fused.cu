// Fused path for one grid: a single persistent cooperative launch runs the
// whole solve.  Each block owns a fixed set of tiles (2-D: tiles of ti x 32
// cells, ti chosen so that every SM gets at most one tile when the grid
// allows: up to 16 rows in static shared memory, up to 64 rows in dynamic
// shared memory; larger grids loop over 16 x 32 tiles, 1-D over 1024-cell
// tiles, each block an even contiguous share of them); the two stages of
// every step are separated by a device-wide barrier that also sums the
// volume moment over the blocks (barrier_sum).
//
// One tile per block: the tile stays in shared memory for the whole solve
// (each stage updates it in place, the stage-2 base values n^k live in
// registers), so between stages only its halo comes from L2.  While thread 0
// waits at the barrier, warps 1-6 compute the next stage's faces that read
// only the tile's own cells and warp 7 reduces the output moments of output
// steps (2-D: the threads' column sums S_p = sum x1^p n, weighted by x2^q dA;
// summed into the rows after the solve).  After the barrier warp 0
// advances the block's private copy of the scalar chain (solute balance,
// kinetics, CFL step, the next stage's coefficients - identical in every
// block) and hands the halo over to warps 1-6 through a named barrier; they
// load it and compute the faces that read it.  Face values are one FMA on the
// Newton-Raphson quotient (psi_quot_fast).
//
// GB300 FP64 notes that shape this kernel: a warp-wide FP64 instruction
// occupies the SM's FP64 pipe for ~16-18 cycles whatever its active lanes,
// and one warp issues about one FP64 instruction per ~64 cycles whether or
// not they depend on each other, so the scalar chain between stages (the
// critical path on small grids) costs about 64 cycles per FP64 instruction
// and is kept short: the moment weights of each thread's cells are computed
// once, the cross-block sum costs no round trip beyond the barrier's own
// (fixed-point warp sums), the stage coefficients are computed once per
// block from registers, the temperature once per step, the kinetics use
// table-driven exp and log, and the second rate evaluation of a step is a
// short series from the first (RateCarry).  The 2-D output moments are
// separable column sums, combined by the moment warp.
//
// Every wait is bounded: a barrier that does not complete within about one
// second sets PBE_ETIMEOUT and the kernel returns.
#include <algorithm>
#include <type_traits>

#include "pbe_chain.cuh"
#include "pbe_internal.h"
#include "pbe_sync.cuh"
#include "pbe_tiles.cuh"

namespace pbe {

constexpr int kFNT = 256;     // threads per block (the reductions assume 256)
constexpr int kFT1 = 1024;    // 1-D tile
constexpr int kFTI = 16;      // 2-D tile height of the multi-tile launch (and the largest of the small one-tile kernel)
constexpr int kFTIBig = 64;   // largest 2-D tile height of the one-tile kernel for larger grids (dynamic shared memory)
constexpr int kFTJ = 32;      // 2-D tile columns

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
// Named barrier 3: warp 0 arrives once the device-wide barrier of the stage
// is done (non-blocking), the face warps wait on it before they load the halo.
// The unaligned forms: warp 0 reaches it after thread 0's wait.
struct HaloGo {
    static __device__ __forceinline__ void arrive() { asm volatile("bar.arrive 3, %0;" ::"r"(32 * (kFaceWarps + 1)) : "memory"); }
    static __device__ __forceinline__ void wait() { asm volatile("bar.sync 3, %0;" ::"r"(32 * (kFaceWarps + 1)) : "memory"); }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

template <int NDIM, int TI>
struct FusedSmem;
template <int TI>
struct FusedSmem<1, TI> {
    double tile[kFT1 + 3];
    double h[kFT1 + 1];
};
template <int TI>
struct FusedSmem<2, TI> {
    Tile2DSmem<TI, kFTJ> t;
};

// cells of one tile (2-D: up to TI rows of 32)
template <int NDIM, int TI>
struct TileShape {
    static constexpr int CELLS = NDIM == 1 ? kFT1 : TI * kFTJ;
};

// the tile's shared memory: static for the kFTI-row tiles, dynamic (set at
// launch) for the taller ones
template <int NDIM, int TI>
__device__ __forceinline__ FusedSmem<NDIM, TI>& fused_smem()
{
    if constexpr (TI > kFTI) {
        extern __shared__ __align__(16) double fused_dyn[];
        return *reinterpret_cast<FusedSmem<NDIM, TI>*>(fused_dyn);
    } else {
        __shared__ FusedSmem<NDIM, TI> sm_static;
        return sm_static;
    }
}

template <int NDIM>
__device__ __forceinline__ void tile_origin(int t, int tiles_x, int ti, int& i0, int& j0)
{
    if (NDIM == 1) { i0 = t * kFT1; j0 = 0; }
    else { i0 = (t / tiles_x) * ti; j0 = (t % tiles_x) * kFTJ; }
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

// Stage a 2-D tile of ti (<= kFTI) rows with its halo and compute every face
// value, on the `nthr` threads whose rank in the group is `tid`.  HALO_ONLY:
// the tile's own cells are already in shared memory and the faces that read
// only them (faces2d_interior) are done; load the halo and compute the faces
// that read it.  The faces read the halo rows at the tile's columns and the
// halo columns at its rows, never the corners.
template <bool HALO_ONLY, int TI, bool MERGE = false, class Sync>
__device__ __forceinline__ void faces2d_rows(const double* in, int i0, int j0, int ti, const Geom& g,
                                             Tile2DSmem<TI, kFTJ>& s, int tid, int nthr, Sync sync)
{
    constexpr int W = kFTJ + 3;
    const int N1 = g.N1, N2 = g.N2;
    if (HALO_ONLY) {
        const int nrow = 3 * kFTJ;   // rows -2, -1, ti at the tile's columns; then columns -2, -1, 32 at its rows
        for (int k = tid; k < nrow + 3 * ti; k += nthr) {
            int r, c;
            if (k < nrow) {
                const int h = k / kFTJ;
                r = h < 2 ? h : ti + 2;
                c = 2 + (k - h * kFTJ);
            } else {
                const int kk = k - nrow, h = kk / ti;
                r = 2 + (kk - h * ti);
                c = h < 2 ? h : kFTJ + 2;
            }
            const int gi = i0 - 2 + r, gj = j0 - 2 + c;
            s.tile[r * W + c] = (gi >= 0 && gi < N1 && gj >= 0 && gj < N2) ? __ldcg(in + (size_t)gi * N2 + gj) : 0.0;
        }
    } else {
        for (int k = tid; k < (ti + 3) * W; k += nthr) {
            const int r = k / W, c = k - r * W;
            const int gi = i0 - 2 + r, gj = j0 - 2 + c;
            s.tile[k] = (gi >= 0 && gi < N1 && gj >= 0 && gj < N2) ? __ldcg(in + (size_t)gi * N2 + gj) : 0.0;
        }
    }
    sync();
    if (HALO_ONLY) {
        // L1 faces 0, 1 and ti of every column, then L2 faces 0, 1 and 32 of every row
        const int nrow = 3 * kFTJ;
        for (int k = tid; k < nrow + 3 * ti; k += nthr) {
            if (k < nrow) {
                const int h = k / kFTJ, c = k - h * kFTJ, f = h < 2 ? h : ti;
                s.h1[f * kFTJ + c] = face_value<true>(s.tile[f * W + c + 2], s.tile[(f + 1) * W + c + 2],
                                                      s.tile[(f + 2) * W + c + 2]);
            } else {
                const int kk = k - nrow, h = kk / ti, r = kk - h * ti, f = h < 2 ? h : kFTJ;
                const double* row = s.tile + (r + 2) * W;
                s.h2[r * (kFTJ + 1) + f] = face_value<true>(row[f], row[f + 1], row[f + 2]);
            }
        }
    } else if (MERGE) {
        // L1 and L2 faces in one index space, so that the ragged last pass runs on
        // two warps at once rather than twice in a row on warp 0
        const int n1f = (ti + 1) * kFTJ;
        for (int k = tid; k < n1f + ti * (kFTJ + 1); k += nthr) {
            if (k < n1f) {
                const int f = k / kFTJ, c = k - f * kFTJ;
                s.h1[k] = face_value<true>(s.tile[f * W + c + 2], s.tile[(f + 1) * W + c + 2], s.tile[(f + 2) * W + c + 2]);
            } else {
                const int kk = k - n1f, r = kk / (kFTJ + 1), f = kk - r * (kFTJ + 1);
                const double* row = s.tile + (r + 2) * W;
                s.h2[kk] = face_value<true>(row[f], row[f + 1], row[f + 2]);
            }
        }
    } else {
        for (int k = tid; k < (ti + 1) * kFTJ; k += nthr) {
            const int f = k / kFTJ, c = k - f * kFTJ;
            s.h1[k] = face_value<true>(s.tile[f * W + c + 2], s.tile[(f + 1) * W + c + 2], s.tile[(f + 2) * W + c + 2]);
        }
        for (int k = tid; k < ti * (kFTJ + 1); k += nthr) {
            const int r = k / (kFTJ + 1), f = k - r * (kFTJ + 1);
            const double* row = s.tile + (r + 2) * W;
            s.h2[k] = face_value<true>(row[f], row[f + 1], row[f + 2]);
        }
    }
}

// The faces of a 2-D tile that read only the tile's own cells (tile rows and
// columns 2 .. ti+1 / 2 .. 33 of the staged array): L1 faces 2 .. ti-1 of
// every column and L2 faces 2 .. 31 of every row.  No memory traffic beyond
// shared memory, so they can run while the device-wide barrier is pending.
template <int TI>
__device__ __forceinline__ void faces2d_interior(int ti, Tile2DSmem<TI, kFTJ>& s, int tid, int nthr)
{
    constexpr int W = kFTJ + 3;
    for (int k = tid; k < (ti - 2) * kFTJ; k += nthr) {
        const int f = 2 + k / kFTJ, c = k % kFTJ;
        s.h1[f * kFTJ + c] = face_value<true>(s.tile[f * W + c + 2], s.tile[(f + 1) * W + c + 2],
                                              s.tile[(f + 2) * W + c + 2]);
    }
    constexpr int NF = kFTJ - 2;
    for (int k = tid; k < ti * NF; k += nthr) {
        const int r = k / NF, f = 2 + (k - r * NF);
        const double* row = s.tile + (r + 2) * W;
        s.h2[r * (kFTJ + 1) + f] = face_value<true>(row[f], row[f + 1], row[f + 2]);
    }
}

template <int NDIM, bool HALO_ONLY, int TI, bool MERGE = false, class Sync>
__device__ __forceinline__ void fused_faces(const double* in, int t, int tiles_x, int ti, const Geom& g,
                                            FusedSmem<NDIM, TI>& sm, int tid, int nthr, Sync sync)
{
    int i0, j0;
    tile_origin<NDIM>(t, tiles_x, ti, i0, j0);
    if constexpr (NDIM == 1) {
        if (HALO_ONLY) {   // cells i0-2, i0-1 and i0+T, then faces 0, 1 and T
            const int N = g.N1;
            if (tid < 3) {
                const int k = tid < 2 ? tid : kFT1 + 2, gi = i0 - 2 + k;
                sm.tile[k] = (gi >= 0 && gi < N) ? __ldcg(in + gi) : 0.0;
            }
            sync();
            if (tid < 3) {
                const int f = tid < 2 ? tid : kFT1;
                sm.h[f] = face_value<true>(sm.tile[f], sm.tile[f + 1], sm.tile[f + 2]);
            }
        } else {
            faces1d<true, true, kFT1>(in, i0, g, sm.tile, sm.h, tid, nthr, sync);
        }
    } else {
        faces2d_rows<HALO_ONLY, TI, MERGE>(in, i0, j0, ti, g, sm.t, tid, nthr, sync);
    }
}

// faces of the block's tile that read only its own cells (one tile per block)
template <int NDIM, int TI>
__device__ __forceinline__ void fused_faces_interior(int ti, FusedSmem<NDIM, TI>& sm, int tid, int nthr)
{
    if constexpr (NDIM == 1) {
        for (int f = 2 + tid; f < kFT1; f += nthr) sm.h[f] = face_value<true>(sm.tile[f], sm.tile[f + 1], sm.tile[f + 2]);
    } else {
        faces2d_interior(ti, sm.t, tid, nthr);
    }
}

// update of cell local index k of tile (i0, j0) from the faces in shared memory.
// ONE_TILE (the block keeps its tile for the whole solve): the stage-2 base
// value n^k comes from the register `keep` (updated here), and the new value
// also replaces the cell's own entry of the shared tile, the next stage's
// input - the faces of this stage are already computed and each thread reads
// only its own cells' entries here.
template <int STAGE, int NDIM, bool ONE_TILE, int TI>
__device__ __forceinline__ double cell_update(const double* old, double* out, int k, int i0, int j0, int ti, const Geom& g,
                                              const StageCoef& sc, FusedSmem<NDIM, TI>& sm, double& keep, bool& valid,
                                              int& i, int& j)
{
    int r, c;
    cell_of<NDIM>(k, i0, j0, i, j, r, c);
    valid = (NDIM == 1) ? (i < g.N1) : (r < ti && i < g.N1 && j < g.N2);
    if (!valid) return 0.0;
    double v;
    size_t gidx;
    double* slot;
    if constexpr (NDIM == 1) {
        slot = sm.tile + r + 2;
        v = *slot + sc.c1 * (sm.h[r] - sm.h[r + 1]);
        gidx = i;
        if (i == 0) v += sc.src;
    } else {
        constexpr int W = kFTJ + 3;
        auto& s = sm.t;
        slot = s.tile + (r + 2) * W + c + 2;
        v = *slot + sc.c1 * (s.h1[r * kFTJ + c] - s.h1[(r + 1) * kFTJ + c]) +
            sc.c2 * (s.h2[r * (kFTJ + 1) + c] - s.h2[r * (kFTJ + 1) + c + 1]);
        gidx = (size_t)i * g.N2 + j;
        if (i == 0 && j == 0) v += sc.src;
    }
    if (STAGE == 2) v = 0.5 * (ONE_TILE ? keep : old[gidx]) + 0.5 * v;
    out[gidx] = v;
    if (ONE_TILE) {
        *slot = v;
        if (STAGE == 2) keep = v;
    }
    return v;
}

template <int NDIM, bool ONE_TILE, int TI>
__global__ void __launch_bounds__(kFNT, 1) k_fused(double* n, double* n1, Scal* S, Kin K, Geom g, double* part,
                                                   const double* t_out, double* rows, unsigned int* bar, int ntiles,
                                                   int tiles_x, int ti, long long wait_limit, double* rowpart)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    constexpr int CPT = TileShape<NDIM, TI>::CELLS / kFNT;   // cells per thread per tile
    static_assert(TI == kFTI || (NDIM == 2 && ONE_TILE), "tall tiles only for the 2-D one-tile kernel");
    __shared__ Scal s;
    __shared__ StageCoef scs;   // coefficients of the coming stage (written by thread 0)
    __shared__ double red[kFNT * (NM + 1)];
    __shared__ double red2[256];
    __shared__ double msum[NM];
    __shared__ int fail;
    FusedSmem<NDIM, TI>& sm = fused_smem<NDIM, TI>();
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
    double* my_rows = blockIdx.x == 0 ? rows : nullptr;
    // the volume moment is summed across blocks in fixed point (barrier_sum):
    // unit u = 2^(E-52) with 2^E above twice the largest volume moment the
    // solute balance allows, V0 + C / kappa (crystals grow only while S > 1),
    // so that an error of u in V moves C by about 2^-52 C
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(bar);
    unsigned long long acc_base0 = 0ull, acc_base1 = 0ull;
    double u, inv_u;
    {
        double vmax = 2.0 * (s.V0 + (K.kappa > 0.0 ? s.C / K.kappa : 0.0));
        if (!(vmax > 0.0) || !isfinite(vmax)) vmax = 1.0;
        const int E = ilogb(vmax) + 1;
        u = ldexp(1.0, E - 52);
        inv_u = ldexp(1.0, 52 - E);
    }
    unsigned int gen = 0;
    // warp 0: the stage-1 chain's evaluation, for the stage-2 chain's series
    // (in shared memory: in registers it would cost the one-tile kernels their
    // second block per SM, which grids of 153-304 tiles need)
    __shared__ RateCarry rcs[32];
    if (warp == 0) rate_carry_init(rcs[threadIdx.x], K);

    // moment weights of this thread's cells (one tile per block: fixed for the
    // whole solve).  1-D: the four weights of each cell in registers.  2-D
    // tiles of up to kFTI rows (two cells a thread): the moments are
    // separable, mu_pq = sum_j x2_j^q dA sum_i x1_i^p n_ij, and a thread's
    // cells lie in one column (tiles are 32 wide), so each thread keeps x1,
    // x1^2, x1^3 of its cells and x2^q dA of its column and sums
    // S_p = sum x1^p v over its cells (four FMAs a cell instead of ten), and
    // the moment warp combines the columns (about 50 FP64 instructions
    // against 90 for the per-thread moments: it was the last warp of the
    // stage on output steps).  Tall tiles (eight cells a thread, measured
    // faster this way): x1 and the volume weight of each cell, x2^q dA of the
    // column, all ten moments a thread.
    constexpr bool WREG = ONE_TILE && NDIM == 1;
    constexpr bool SEP = ONE_TILE && NDIM == 2 && TI <= kFTI;
    constexpr bool WCOL = ONE_TILE && NDIM == 2 && !SEP;
    static_assert(!SEP || kFNT - 32 * (kFaceWarps + 1) == 32, "one moment warp");
    double wgt[WREG ? CPT : 1][WREG ? NM : 1];
    double x1p[SEP ? CPT : 1][3];
    double x1c[WCOL ? CPT : 1], w8c[WCOL ? CPT : 1];
    double wx2[4] = {0.0, 0.0, 0.0, 0.0};   // x2^q dA of this thread's column
    double keep[ONE_TILE ? CPT : 1];   // n at the start of the step for this thread's cells
    keep[0] = 0.0;
    if constexpr (ONE_TILE) {
        int i0, j0;
        tile_origin<NDIM>(blockIdx.x, tiles_x, ti, i0, j0);
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            int i, j, r, c;
            cell_of<NDIM>(threadIdx.x + q * kFNT, i0, j0, i, j, r, c);
            if constexpr (SEP || WCOL) {
                const double x2 = (j + 0.5) * g.d2, a = g.d1 * g.d2;
                wx2[0] = a; wx2[1] = a * x2; wx2[2] = wx2[1] * x2; wx2[3] = wx2[2] * x2;
                const double x1 = (i + 0.5) * g.d1;
                if constexpr (SEP) {
                    x1p[q][0] = x1; x1p[q][1] = x1 * x1; x1p[q][2] = x1p[q][1] * x1;
                } else {
                    x1c[q] = x1;
                    w8c[q] = x1 * wx2[2];
                }
            } else {
                moment_weights<NDIM>(i, j, g, wgt[q]);
            }
            const bool valid = (NDIM == 1) ? (i < g.N1) : (r < ti && i < g.N1 && j < g.N2);
            keep[q] = valid && (int)blockIdx.x < ntiles ? n[(size_t)i * g.N2 + j] : 0.0;
        }
    }

    // this block's tiles: blockIdx.x (if below ntiles) with ONE_TILE; otherwise
    // an even contiguous share, so that every SM gets ntiles / SMs tiles to within one
    // whichever way consecutive blocks are placed on the SMs (round-robin strides
    // gave the first blocks one tile more, and those share SMs)
    const int t_first = ONE_TILE ? (int)blockIdx.x : (int)(((long long)blockIdx.x * ntiles) / G);
    const int t_end = ONE_TILE ? ntiles : (int)(((long long)(blockIdx.x + 1) * ntiles) / G);
    const int t_step = ONE_TILE ? G : 1;
    fused_faces<NDIM, false, TI, !ONE_TILE>(n, t_first, tiles_x, ti, g, sm, threadIdx.x, kFNT, BlockSync());
    __syncthreads();
    for (;;) {
        // temperature and solubility at the end of this step: both kinetics of
        // the step are evaluated there (warp 0, once per step)
        KinT tpre{0.0, 0.0};
        if (warp == 0 && K.kind != PBE_KINETICS_FIXED) tpre = kin_temperature(K, s.t_new);
#pragma unroll 1
        for (int stage = 1; stage <= 2; ++stage) {
            const StageCoef sc = scs;
            const double* in = stage == 1 ? n : n1;
            double* out = stage == 1 ? n1 : n;
            double m[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) m[k] = 0.0;
            // several tiles a block, volume moment only (no output step): mv = V / dL
            // (1-D: sum x^3 v) or V / (dL1 dL2) (2-D: sum over tiles of x2^2 sum_q x1 v),
            // from per-tile bases - the thread's cells of a tile lie kFNT apart in 1-D
            // and in one column, 8 rows apart, in 2-D
            const bool vol_only = !ONE_TILE && !sc.moms;
            double mv = 0.0;
            for (int t = t_first; t < t_end; t += t_step) {
                if (t != t_first) {
                    fused_faces<NDIM, false, TI, !ONE_TILE>(in, t, tiles_x, ti, g, sm, threadIdx.x, kFNT, BlockSync());
                    __syncthreads();
                }
                int i0, j0;
                tile_origin<NDIM>(t, tiles_x, ti, i0, j0);
                if (!ONE_TILE && vol_only) {
                    static_assert(ONE_TILE || NDIM == 1 || (TI * kFTJ == 2 * kFNT && kFNT % kFTJ == 0),
                                  "2-D multi-tile cells: two a thread, 8 rows apart in one column");
                    double acc = 0.0;
                    const double xb = NDIM == 1 ? (i0 + (int)threadIdx.x + 0.5) * g.d1
                                                : (i0 + warp + 0.5) * g.d1;
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        bool valid;
                        int i, j;
                        double& kq = keep[0];
                        const double v = stage == 1
                            ? cell_update<1, NDIM, ONE_TILE, TI>(n, out, threadIdx.x + q * kFNT, i0, j0, ti, g, sc, sm, kq, valid, i, j)
                            : cell_update<2, NDIM, ONE_TILE, TI>(n, out, threadIdx.x + q * kFNT, i0, j0, ti, g, sc, sm, kq, valid, i, j);
                        // invalid cells return 0 and add nothing
                        if (NDIM == 1) {
                            const double x = q == 0 ? xb : fma((double)(q * kFNT), g.d1, xb);
                            acc = fma(x * x * x, v, acc);
                        } else {
                            const double x1 = q == 0 ? xb : fma((double)(q * (kFNT / kFTJ)), g.d1, xb);
                            acc = fma(x1, v, acc);
                        }
                    }
                    if (NDIM == 1) {
                        mv += acc;
                    } else {
                        const double x2 = (j0 + (int)(threadIdx.x & 31) + 0.5) * g.d2;
                        mv = fma(x2 * x2, acc, mv);
                    }
                    __syncthreads();
                    continue;
                }
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    bool valid;
                    int i, j;
                    double& kq = keep[ONE_TILE ? q : 0];
                    const double v = stage == 1
                        ? cell_update<1, NDIM, ONE_TILE, TI>(n, out, threadIdx.x + q * kFNT, i0, j0, ti, g, sc, sm, kq, valid, i, j)
                        : cell_update<2, NDIM, ONE_TILE, TI>(n, out, threadIdx.x + q * kFNT, i0, j0, ti, g, sc, sm, kq, valid, i, j);
                    if (!valid) continue;
                    if constexpr (SEP) {   // m[p] = S_p of the thread's column
                        if (sc.moms) {
                            m[0] += v;
                            m[1] = fma(x1p[q][0], v, m[1]);
                            m[2] = fma(x1p[q][1], v, m[2]);
                            m[3] = fma(x1p[q][2], v, m[3]);
                        } else {
                            m[1] = fma(x1p[q][0], v, m[1]);
                        }
                        continue;
                    }
                    if constexpr (WCOL) {
                        if (sc.moms) {
                            const double x1 = x1c[q], v1 = x1 * v, v2 = x1 * v1, v3 = x1 * v2;
                            m[0] = fma(wx2[0], v, m[0]);  m[1] = fma(wx2[0], v1, m[1]); m[2] = fma(wx2[1], v, m[2]);
                            m[3] = fma(wx2[0], v2, m[3]); m[4] = fma(wx2[1], v1, m[4]); m[5] = fma(wx2[2], v, m[5]);
                            m[6] = fma(wx2[0], v3, m[6]); m[7] = fma(wx2[1], v2, m[7]); m[8] = fma(wx2[2], v1, m[8]);
                            m[9] = fma(wx2[3], v, m[9]);
                        } else {
                            m[VIDX] = fma(w8c[q], v, m[VIDX]);
                        }
                        continue;
                    }
                    double wl[NM];
                    if constexpr (WREG) {
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
            if (vol_only) m[VIDX] = mv * (NDIM == 1 ? g.d1 : g.d1 * g.d2);
            const int row_here = s.out_idx;
            // only the volume moment is on the critical path; on output steps
            // the per-thread moments wait in shared memory and are reduced
            // while the barrier is pending, the row completed after the solve
            if constexpr (SEP) {
                if (sc.moms) {
#pragma unroll
                    for (int p = 0; p < 4; ++p) red[p * kFNT + threadIdx.x] = m[p];
                }
                m[VIDX] = wx2[2] * m[1];   // mu_12 = x2^2 dA sum x1 v
            } else if (sc.moms) {
#pragma unroll
                for (int k = 0; k < NM; ++k) red[threadIdx.x * (NM + 1) + k] = m[k];
            }
            const long long qb = block_sum_fixed_t0(m[VIDX], inv_u, reinterpret_cast<long long*>(red2));
            if (warp == 0) {
                if (threadIdx.x == 0) {
                    double total = 0.0;
                    const int p = (int)(gen & 1u);
                    unsigned long long base = p ? acc_base1 : acc_base0;
                    const bool ok = barrier_sum(acc + p * kAccStride, base, qb, u, (unsigned int)G, wait_limit, total);
                    if (p) acc_base1 = base;
                    else acc_base0 = base;
                    msum[VIDX] = total;
                    fail = !ok;
                }
                __syncwarp();
                HaloGo::arrive();   // the other blocks' outputs are visible: the face warps may load the halo
                if (!fail) {
                    // the next stage's coefficients, once per block (the divisions of
                    // stage_coef in every thread cost the FP64 pipe ~4k cycles a stage)
                    const StageCoef c = stage == 1 ? fused_finish1<false, true>(&s, K, g, msum[VIDX], tpre, &rcs[threadIdx.x & 31])
                                                   : fused_finish2<false, true>(&s, K, g, t_out, my_rows, msum, NM, VIDX, tpre, &rcs[threadIdx.x & 31]);
                    if (threadIdx.x == 0) scs = c;
                }
            } else if (warp <= kFaceWarps) {
                // one tile per block: the next stage's input is already in shared
                // memory except the halo, and its faces that do not read the halo
                // need nothing from the other blocks - computed while the barrier
                // is pending; then the halo and the faces that read it
                if (ONE_TILE) fused_faces_interior<NDIM, TI>(ti, sm, threadIdx.x - 32, 32 * kFaceWarps);
                HaloGo::wait();
                if (!fail)
                    fused_faces<NDIM, ONE_TILE, TI, !ONE_TILE>(stage == 1 ? n1 : n, t_first, tiles_x, ti, g, sm,
                                                    threadIdx.x - 32, 32 * kFaceWarps, GroupSync());
            } else if (SEP && sc.moms) {
                // the block's ten moments from the column sums S_p: lane c sums its
                // column over the eight warps, weights it with x2_c^q dA (its own
                // column's weights), and a transposed butterfly sums the columns
                const int lane = threadIdx.x & 31;
                double T[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const double* rp = red + p * kFNT + lane;
                    T[p] = ((rp[0] + rp[32]) + (rp[64] + rp[96])) + ((rp[128] + rp[160]) + (rp[192] + rp[224]));
                }
                const double mu[10] = {wx2[0] * T[0], wx2[0] * T[1], wx2[1] * T[0], wx2[0] * T[2], wx2[1] * T[1],
                                       wx2[2] * T[0], wx2[0] * T[3], wx2[1] * T[2], wx2[2] * T[1], wx2[3] * T[0]};
                int idx;
                const double tot = transposed_sum10(mu, lane, idx);
                if ((lane & 1) == 0 && idx < NM) rowpart[((size_t)row_here * G + blockIdx.x) * NM + idx] = tot;
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
            gen += 1u;
            __syncthreads();
            if (fail) break;
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
// (one block per row, one warp per moment: lane-strided partial sums, then a
// butterfly; a fixed order, so the rows are the same on every run).
template <int NDIM>
__global__ void k_fused_rows(const double* rowpart, int G, const Scal* S, double* rows)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    const int r = S->row_first + blockIdx.x;
    const int m = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (r >= S->out_idx || m >= NM) return;
    double acc = 0.0;
    for (int b = lane; b < G; b += 32) acc += rowpart[((size_t)r * G + b) * NM + m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rows[(size_t)r * (NM + 2) + 1 + m] = acc;
}

// Tiles of the fused launch: 1-D 1024 cells; 2-D ti x 32 with the smallest
// ti (>= 4) that gives every co-resident block at most one tile (all SMs
// busy, fewer cells each) - ti <= kFTI in the small-tile kernel, up to
// kFTIBig in the tall-tile one (*tall) - else kFTI x 32 tiles looped over.
static int fused_tiles(const Geom& g, int max_blocks, int* tiles_x, int* ti, bool* tall)
{
    *tall = false;
    if (g.ndim == 1) {
        *tiles_x = 1;
        *ti = 1;
        return (g.N1 + kFT1 - 1) / kFT1;
    }
    *tiles_x = (g.N2 + kFTJ - 1) / kFTJ;
    *ti = kFTI;
    if (*tiles_x <= max_blocks) {
        const int rows_of_tiles = max_blocks / *tiles_x;
        int t = (g.N1 + rows_of_tiles - 1) / rows_of_tiles;
        if (t < 4) t = 4;
        if (t <= kFTI) {
            *ti = t;
        } else if (t <= kFTIBig) {
            *ti = t;
            *tall = true;
        }
    }
    return *tiles_x * ((g.N1 + *ti - 1) / *ti);
}

bool fused_supported(const pbe_grid* g) { return g->d_bar != nullptr; }

// Blocks, tiles and kernel of the fused launch of a grid (depends only on the
// geometry and the device: computed once per grid).
static cudaError_t fused_config(pbe_grid* g)
{
    if (g->fused_fn) return cudaSuccess;
    const int sms = g->sms;
    // blocks the launch may use: one per SM, at most max_blocks / 2 (the row
    // partials' store) and the grid's block limit
    int lim = std::min(sms, g->max_blocks / 2);
    if (g->block_limit > 0) lim = std::min(lim, g->block_limit);
    int tiles_x, ti;
    bool tall;
    int ntiles = fused_tiles(g->geo, lim, &tiles_x, &ti, &tall);
    const void* fn_multi = g->geo.ndim == 1 ? (const void*)k_fused<1, false, kFTI> : (const void*)k_fused<2, false, kFTI>;
    const void* fn_one = g->geo.ndim == 1 ? (const void*)k_fused<1, true, kFTI>
                                          : (tall ? (const void*)k_fused<2, true, kFTIBig> : (const void*)k_fused<2, true, kFTI>);
    const size_t dyn = tall ? sizeof(FusedSmem<2, kFTIBig>) : 0;
    cudaError_t e;
    if (tall && (e = cudaFuncSetAttribute(fn_one, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) != cudaSuccess)
        return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn_one, kFNT, dyn);
    if (e != cudaSuccess) return e;
    int G = ntiles;
    if (G > occ * sms) G = occ * sms;
    if (2 * G > g->max_blocks) G = g->max_blocks / 2;
    if (g->block_limit > 0 && G > g->block_limit) G = g->block_limit;
    if (G < 1) G = 1;
    if (G > 1000) G = 1000;   // the arrival count of barrier_sum has 10 bits
    const void* fn = fn_one;
    size_t fn_dyn = dyn;
    if (G < ntiles && g->geo.ndim == 2 && g->window_mode != 0) {
        // more tiles than co-resident blocks on a large 2-D grid: the persistent
        // window kernel (no halo faces recomputed per 16 x 32 tile)
        FusedWinCfg c;
        e = fused_window_config(g->geo, sms, g->block_limit > 0 ? std::min(g->max_blocks / 2, g->block_limit)
                                                                : g->max_blocks / 2, &c);
        if (e != cudaSuccess) return e;
        g->fused_blocks = c.G;
        g->fused_ntiles = c.ntiles;
        g->fused_tiles_x = c.tiles_x;
        g->fused_ti = c.ti;
        g->fused_dyn = c.dyn;
        g->fused_fn = c.fn;
        return cudaSuccess;
    }
    if (G < ntiles) {   // more tiles than co-resident blocks: kFTI x 32 tiles looped over
        fn = fn_multi;
        fn_dyn = 0;
        if (g->geo.ndim == 2) {
            ti = kFTI;
            ntiles = tiles_x * ((g->geo.N1 + kFTI - 1) / kFTI);
        }
        int occ2 = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, fn_multi, kFNT, 0);
        if (e != cudaSuccess) return e;
        // at most two blocks per SM: measured on GB300, 1-D 2^20 cells 31.2 / 28.0 /
        // 29.1 ms and 2^19 9.3 / 8.3 / 8.6 ms at one / two / three blocks per SM
        // (three add barrier arrivals and pile more tiles on the busiest SM)
        G = std::min(ntiles, std::min(occ2, 2) * sms);
        if (2 * G > g->max_blocks) G = g->max_blocks / 2;
        if (g->block_limit > 0 && G > g->block_limit) G = g->block_limit;
        if (G < 1) G = 1;
        if (G > 1000) G = 1000;
    }
    g->fused_blocks = G;
    g->fused_ntiles = ntiles;
    g->fused_tiles_x = tiles_x;
    g->fused_ti = ti;
    g->fused_dyn = fn_dyn;
    g->fused_fn = fn;
    return cudaSuccess;
}

cudaError_t launch_fused_solve(pbe_grid* g, int n_out)
{
    cudaError_t e = fused_config(g);
    if (e != cudaSuccess) return e;
    const int G = g->fused_blocks;
    int ntiles = g->fused_ntiles, tiles_x = g->fused_tiles_x, ti = g->fused_ti;
    const void* fn = g->fused_fn;
    e = cudaMemsetAsync(g->d_bar, 0, 2 * kAccStride * sizeof(unsigned long long), g->stream);
    if (e != cudaSuccess) return e;
    long long wait_limit = g->wait_cycles > 0 ? g->wait_cycles : (g->wait_cycles == 0 ? 0 : kBarrierCycles);
    void* args[] = {&g->d_n, &g->d_n1, &g->d_S, &g->kin, &g->geo, &g->d_part, &g->d_tout, &g->d_rows,
                    &g->d_bar, (void*)&ntiles, &tiles_x, &ti, &wait_limit, &g->d_rowpart};
    if (g->timing && (e = cudaEventRecord(g->ev_k0, g->stream)) != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel(fn, G, kFNT, args, g->fused_dyn, g->stream);
    if (e != cudaSuccess) return e;
    if (g->timing && (e = cudaEventRecord(g->ev_k1, g->stream)) != cudaSuccess) return e;
    const int nrows = n_out > 0 ? n_out : 1;
    if (g->geo.ndim == 1) k_fused_rows<1><<<nrows, 4 * 32, 0, g->stream>>>(g->d_rowpart, G, g->d_S, g->d_rows);
    else k_fused_rows<2><<<nrows, 10 * 32, 0, g->stream>>>(g->d_rowpart, G, g->d_S, g->d_rows);
    return cudaGetLastError();
}

}  // namespace pbe
