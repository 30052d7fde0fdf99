// Device-wide synchronization of the persistent cooperative kernels: a
// barrier over the co-resident blocks that also sums one value exactly
// (fixed point, independent of the arrival order), and the block sum in
// that fixed-point unit.
#pragma once

#include "pbe_device.cuh"

namespace pbe {

constexpr long long kBarrierCycles = 2000000000LL;  // default wait limit: ~1 s at 2 GHz

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long atom_add_release_u64(unsigned long long* p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

// Device-wide barrier over the co-resident blocks of the cooperative launch
// that also sums one value over the blocks, exactly and independently of the
// arrival order (so every block, on every run, gets the same total): each
// block adds its value, an integer multiple q of the unit u (a power of
// two), as (q << 10) + 1, to a 64-bit accumulator with a release
// add (cumulative over the writes the block barrier ordered before it), and
// waits with acquire loads.  The low 10 bits count the arrivals of the
// stage, the rest sums q (integer addition is associative; the accumulator
// wraps modulo 2^64, differences stay exact).  Stages alternate between two
// accumulators (a block cannot reach stage s+2 before every block has read
// stage s).  Thread 0 only; returns false when the wait runs past `limit`
// cycles.
constexpr int kAccStride = 16;   // the two accumulators lie 128 bytes apart
__device__ inline bool barrier_sum(unsigned long long* acc, unsigned long long& base, long long q, double u,
                            unsigned int nblocks, long long limit, double& total)
{
    atom_add_release_u64(acc, ((unsigned long long)q << 10) + 1ull);
    unsigned long long x = ld_acquire_u64(acc);
    if (((x - base) & 1023ull) != nblocks) {
        const long long t0 = clock64();
        const unsigned int spin = limit > 0 ? 64u : 1u;
        for (unsigned int polls = 0;;) {
            x = ld_acquire_u64(acc);
            if (((x - base) & 1023ull) == nblocks) break;
            if (++polls > spin) {
                if (clock64() - t0 > limit) return false;
                __nanosleep(20);
            }
        }
    }
    const long long sq = (long long)(x - base - nblocks) >> 10;
    base = x;
    total = (double)sq * u;
    return true;
}

// Block sum of one value (256 threads) in the fixed-point unit of
// barrier_sum, for thread 0 only: every thread rounds its value to a
// multiple q of u, each warp adds its q exactly with two 32-bit reductions
// (the low 26 bits and the rest of q), and thread 0 adds the eight warp
// sums.  Integer adds leave the FP64 pipe to the other warps and make the
// sum independent of the order.  |q| < 2^51 (the unit bounds the volume
// moment by 2^52 u) keeps the reduced high parts inside 32 bits.
__device__ __forceinline__ long long block_sum_fixed_t0(double v, double inv_u, long long* wsum)
{
    const long long q = llrint(v * inv_u);
    const int hs = __reduce_add_sync(0xffffffffu, (int)(q >> 26));
    const unsigned ls = __reduce_add_sync(0xffffffffu, (unsigned)(q & 0x3ffffffLL));
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = (long long)hs * (1LL << 26) + (long long)ls;
    __syncthreads();
    return ((wsum[0] + wsum[1]) + (wsum[2] + wsum[3])) + ((wsum[4] + wsum[5]) + (wsum[6] + wsum[7]));
}

}  // namespace pbe
