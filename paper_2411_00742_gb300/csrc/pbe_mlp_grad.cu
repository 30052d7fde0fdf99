// Weight gradient of the learned closure (the training kernel of the hybrid
// model of Sec. 4.2) over many recorded network evaluations at once.
//
// The adjoint records, for every closure evaluation it differentiates, one
// row (x0, x1, x2, lo0, lo1, lo2): the network's inputs and the adjoints of
// its three outputs.  The gradient of sum_r lo_r . o(x_r) with respect to the
// weights is a contraction over those rows:
//   z1 = W1 x + b1, a1 = silu(z1);  z2 = W2 a1 + b2, a2 = silu(z2);
//   la2 = W3^T lo, lz2 = la2 silu'(z2);  la1 = W2^T lz2, lz1 = la1 silu'(z1);
//   dW3 = sum lo a2^T, db3 = sum lo;  dW2 = sum lz2 a1^T, db2 = sum lz2;
//   dW1 = sum lz1 x^T, db1 = sum lz1.
// The three 64-wide products (z2, la1 and dW2, the last one reducing over the
// rows) run on the tensor cores: mma.sync m16n8k16 with bf16 operands and
// fp32 accumulation.  The weights are stored in bf16 already; an activation
// operand is split into two bf16 parts, hi = bf16(v), lo = bf16(v - hi), and
// multiplied by both (dW2, whose operands are both activations: hi.hi +
// hi.lo + lo.hi), so every product keeps about 16 significant bits.  The rest
// (layer 1 and 3, 3-wide) runs on the CUDA cores in fp32.  Each block handles
// a contiguous range of rows in tiles of 64 and writes its partial gradient;
// a second kernel sums the partials in block order (deterministic).
#include <cuda_bf16.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pbe_internal.h"

namespace pbe {

constexpr int kGT = 64;        // rows per tile
constexpr int kGNT = 128;      // threads per block: 4 warps, 16 rows each
constexpr int kMaxGradBlocks = 152;

__device__ __forceinline__ float silu_g(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_g(float z)
{
    const float sg = 1.0f / (1.0f + __expf(-z));
    return sg * (1.0f + z * (1.0f - sg));
}

// two bf16 packed in a 32-bit register, the first in the low half
__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo_half, __nv_bfloat16 hi_half)
{
    return (unsigned)__bfloat16_as_ushort(lo_half) | ((unsigned)__bfloat16_as_ushort(hi_half) << 16);
}

// v = hi + lo in bf16
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// D += A B for one 16x8x16 tile: A 16x16 bf16 (row-major fragment, 4
// registers), B 16x8 bf16 (column fragment, 2 registers), D 16x8 fp32.
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4):
//   A[16][16]: reg0 = A[g][2t..2t+1], reg1 = A[g+8][2t..2t+1],
//              reg2 = A[g][2t+8..2t+9], reg3 = A[g+8][2t+8..2t+9];
//   B[16][8] (k x n): reg0 = B[2t..2t+1][g], reg1 = B[2t+8..2t+9][g];
//   C[16][8]: c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1].
// A fragment from a row-major fp32 matrix M (leading dimension ld) at rows
// r0.., columns k0.., split into hi and lo parts.
__device__ __forceinline__ void frag_a_split(const float* M, int ld, int r0, int k0, unsigned (&hi)[4],
                                             unsigned (&lo)[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int rr[4] = {g, g + 8, g, g + 8}, cc[4] = {2 * t, 2 * t, 2 * t + 8, 2 * t + 8};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float* p = M + (size_t)(r0 + rr[q]) * ld + k0 + cc[q];
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(p[0], h0, l0);
        split_bf16(p[1], h1, l1);
        hi[q] = pack_bf16(h0, h1);
        lo[q] = pack_bf16(l0, l1);
    }
}

// A fragment of the transpose of a row-major fp32 matrix M: A[i][k] = M[k0 + k][r0 + i].
__device__ __forceinline__ void frag_at_split(const float* M, int ld, int r0, int k0, unsigned (&hi)[4],
                                              unsigned (&lo)[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int rr[4] = {g, g + 8, g, g + 8}, cc[4] = {2 * t, 2 * t, 2 * t + 8, 2 * t + 8};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float v0 = M[(size_t)(k0 + cc[q]) * ld + r0 + rr[q]];
        const float v1 = M[(size_t)(k0 + cc[q] + 1) * ld + r0 + rr[q]];
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(v0, h0, l0);
        split_bf16(v1, h1, l1);
        hi[q] = pack_bf16(h0, h1);
        lo[q] = pack_bf16(l0, l1);
    }
}

// B fragment (k x n) with B[k][n] = M[k0 + k][n0 + n] of a row-major fp32 matrix, split.
__device__ __forceinline__ void frag_b_split(const float* M, int ld, int k0, int n0, unsigned (&hi)[2],
                                             unsigned (&lo)[2])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int k = k0 + 2 * t + 8 * q;
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(M[(size_t)k * ld + n0 + g], h0, l0);
        split_bf16(M[(size_t)(k + 1) * ld + n0 + g], h1, l1);
        hi[q] = pack_bf16(h0, h1);
        lo[q] = pack_bf16(l0, l1);
    }
}

// B fragment with B[k][n] = W[n0 + n][k0 + k] of a row-major bf16 matrix (exact).
__device__ __forceinline__ void frag_b_wt(const __nv_bfloat16* W, int ld, int k0, int n0, unsigned (&b)[2])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const __nv_bfloat16* p = W + (size_t)(n0 + g) * ld + k0 + 2 * t + 8 * q;
        b[q] = pack_bf16(p[0], p[1]);
    }
}

// B fragment with B[k][n] = W[k0 + k][n0 + n] of a row-major bf16 matrix (exact).
__device__ __forceinline__ void frag_b_w(const __nv_bfloat16* W, int ld, int k0, int n0, unsigned (&b)[2])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int k = k0 + 2 * t + 8 * q;
        b[q] = pack_bf16(W[(size_t)k * ld + n0 + g], W[(size_t)(k + 1) * ld + n0 + g]);
    }
}

// shared memory of one block (dynamic)
struct GradSm {
    __nv_bfloat16 W2[kMlpH * kMlpH];
    float W1[kMlpH * 3], W3[3 * kMlpH], b1[kMlpH], b2[kMlpH];
    float x[kGT][3], lo[kGT][3];
    float a1[kGT * kMlpH];    // silu(z1)
    float sz1[kGT * kMlpH];   // silu'(z1)
    float a2[kGT * kMlpH];    // silu(z2)
    float lz2[kGT * kMlpH];   // dL/dz2
    float lz1[kGT * kMlpH];   // dL/dz1
};

// offsets of the flat weight layout W1[64][3], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]
constexpr int kOffB1 = kMlpH * 3, kOffW2 = kOffB1 + kMlpH, kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH, kOffB3 = kOffW3 + 3 * kMlpH;
// entries computed on the CUDA cores, per tile: dW1 (192), db1 (64), db2 (64), dW3 (192), db3 (3)
constexpr int kSmallGrads = kMlpH * 3 + kMlpH + kMlpH + 3 * kMlpH + 3;
constexpr int kSmallPerThread = (kSmallGrads + kGNT - 1) / kGNT;

// flat index of small-gradient entry e (0 .. kSmallGrads)
__device__ __forceinline__ int small_index(int e)
{
    if (e < kMlpH * 4) return e;                      // dW1 and db1: indices 0 .. 255
    if (e < kMlpH * 5) return kOffB2 + (e - kMlpH * 4);   // db2
    return kOffW3 + (e - kMlpH * 5);                  // dW3 then db3
}

__global__ void __launch_bounds__(kGNT) k_mlp_grad(const float* __restrict__ rows, long long R,
                                                  const __nv_bfloat16* __restrict__ mW, const float* __restrict__ mB,
                                                  float* __restrict__ part)
{
    extern __shared__ __align__(16) unsigned char gsm_raw[];
    GradSm& s = *reinterpret_cast<GradSm*>(gsm_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    for (int k = tid; k < kMlpH * kMlpH; k += kGNT) s.W2[k] = mW[kMlpH * 3 + k];
    for (int k = tid; k < kMlpH * 3; k += kGNT) {
        s.W1[k] = __bfloat162float(mW[k]);
        s.W3[k] = __bfloat162float(mW[kMlpH * 3 + kMlpH * kMlpH + k]);
    }
    for (int k = tid; k < kMlpH; k += kGNT) { s.b1[k] = mB[k]; s.b2[k] = mB[kMlpH + k]; }
    const long long ntile = (R + kGT - 1) / kGT;
    const long long tf = ntile * blockIdx.x / gridDim.x, te = ntile * (blockIdx.x + 1) / gridDim.x;
    float accW2[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
        for (int q = 0; q < 4; ++q) accW2[n][q] = 0.0f;
    float small[kSmallPerThread];
#pragma unroll
    for (int q = 0; q < kSmallPerThread; ++q) small[q] = 0.0f;
    const int rw = 16 * warp;   // this warp's rows of the tile (and its m-tile of dW2)
    for (long long tl = tf; tl < te; ++tl) {
        const long long r0 = tl * kGT;
        __syncthreads();   // the previous tile's shared arrays are read
        for (int k = tid; k < kGT * 6; k += kGNT) {
            const int r = k / 6, c = k - 6 * r;
            const float v = r0 + r < R ? rows[(size_t)(r0 + r) * 6 + c] : 0.0f;
            if (c < 3) s.x[r][c] = v;
            else s.lo[r][c - 3] = v;
        }
        __syncthreads();
        // layer 1 on the CUDA cores
        for (int k = tid; k < kGT * kMlpH; k += kGNT) {
            const int r = k / kMlpH, h = k - kMlpH * r;
            float z = s.b1[h];
            z = fmaf(s.W1[h * 3], s.x[r][0], z);
            z = fmaf(s.W1[h * 3 + 1], s.x[r][1], z);
            z = fmaf(s.W1[h * 3 + 2], s.x[r][2], z);
            s.a1[k] = silu_g(z);
            s.sz1[k] = silu_grad_g(z);
        }
        __syncthreads();
        // z2 = a1 W2^T on the tensor cores (a1 split in two bf16 parts)
        float acc[8][4];
#pragma unroll
        for (int n = 0; n < 8; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[n][q] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            unsigned ah[4], al[4];
            frag_a_split(s.a1, kMlpH, rw, 16 * ks, ah, al);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                unsigned b[2];
                frag_b_wt(s.W2, kMlpH, 16 * ks, 8 * n, b);
                mma16816(acc[n], ah, b);
                mma16816(acc[n], al, b);
            }
        }
        // a2 = silu(z2), la2 = W3^T lo, lz2 = la2 silu'(z2) at this thread's fragment entries
#pragma unroll
        for (int n = 0; n < 8; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = rw + g + 8 * (q >> 1), h = 8 * n + 2 * t + (q & 1);
                const float z = acc[n][q] + s.b2[h];
                const float la2 = s.W3[h] * s.lo[r][0] + s.W3[kMlpH + h] * s.lo[r][1] + s.W3[2 * kMlpH + h] * s.lo[r][2];
                s.a2[r * kMlpH + h] = silu_g(z);
                s.lz2[r * kMlpH + h] = la2 * silu_grad_g(z);
            }
        __syncthreads();
        // la1 = lz2 W2 on the tensor cores, lz1 = la1 silu'(z1)
#pragma unroll
        for (int n = 0; n < 8; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[n][q] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            unsigned ah[4], al[4];
            frag_a_split(s.lz2, kMlpH, rw, 16 * ks, ah, al);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                unsigned b[2];
                frag_b_w(s.W2, kMlpH, 16 * ks, 8 * n, b);
                mma16816(acc[n], ah, b);
                mma16816(acc[n], al, b);
            }
        }
#pragma unroll
        for (int n = 0; n < 8; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = rw + g + 8 * (q >> 1), j = 8 * n + 2 * t + (q & 1);
                s.lz1[r * kMlpH + j] = acc[n][q] * s.sz1[r * kMlpH + j];
            }
        // dW2 += lz2^T a1 over the tile's rows (both split: hi.hi + hi.lo + lo.hi)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            unsigned ah[4], al[4];
            frag_at_split(s.lz2, kMlpH, rw, 16 * ks, ah, al);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                unsigned bh[2], bl[2];
                frag_b_split(s.a1, kMlpH, 16 * ks, 8 * n, bh, bl);
                mma16816(accW2[n], ah, bh);
                mma16816(accW2[n], ah, bl);
                mma16816(accW2[n], al, bh);
            }
        }
        __syncthreads();
        // the 3-wide layers' gradients and the biases on the CUDA cores, rows in order
#pragma unroll
        for (int q = 0; q < kSmallPerThread; ++q) {
            const int e = tid + q * kGNT;
            if (e >= kSmallGrads) break;
            float a = 0.0f;
            if (e < kMlpH * 3) {                      // dW1[h][k] = sum lz1[r][h] x[r][k]
                const int h = e / 3, k = e - 3 * h;
                for (int r = 0; r < kGT; ++r) a = fmaf(s.lz1[r * kMlpH + h], s.x[r][k], a);
            } else if (e < kMlpH * 4) {               // db1[h] = sum lz1[r][h]
                const int h = e - kMlpH * 3;
                for (int r = 0; r < kGT; ++r) a += s.lz1[r * kMlpH + h];
            } else if (e < kMlpH * 5) {               // db2[h] = sum lz2[r][h]
                const int h = e - kMlpH * 4;
                for (int r = 0; r < kGT; ++r) a += s.lz2[r * kMlpH + h];
            } else if (e < kMlpH * 8) {               // dW3[m][h] = sum lo[r][m] a2[r][h]
                const int m = (e - kMlpH * 5) / kMlpH, h = (e - kMlpH * 5) - kMlpH * m;
                for (int r = 0; r < kGT; ++r) a = fmaf(s.lo[r][m], s.a2[r * kMlpH + h], a);
            } else {                                  // db3[m] = sum lo[r][m]
                const int m = e - kMlpH * 8;
                for (int r = 0; r < kGT; ++r) a += s.lo[r][m];
            }
            small[q] += a;
        }
    }
    // this block's partial gradient in the flat weight layout
    float* out = part + (size_t)blockIdx.x * kMlpNW;
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int h = rw + g + 8 * (q >> 1), j = 8 * n + 2 * t + (q & 1);
            out[kOffW2 + h * kMlpH + j] = accW2[n][q];
        }
#pragma unroll
    for (int q = 0; q < kSmallPerThread; ++q) {
        const int e = tid + q * kGNT;
        if (e < kSmallGrads) out[small_index(e)] = small[q];
    }
}

// dW[e] = sum over the blocks' partials, in block order, in fp64
__global__ void k_mlp_grad_reduce(const float* __restrict__ part, int G, double* __restrict__ dW)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kMlpNW) return;
    double a = 0.0;
    for (int b = 0; b < G; ++b) a += (double)part[(size_t)b * kMlpNW + e];
    dW[e] = a;
}

}  // namespace pbe

namespace pbe {

int mlp_grad_part_floats() { return kMaxGradBlocks * kMlpNW; }

// dW (DEVICE, kMlpNW doubles) = the closure's weight gradient over R rows
// (DEVICE, 6 floats each); part: DEVICE workspace of mlp_grad_part_floats().
cudaError_t launch_mlp_grad(const float* rows, long long R, const __nv_bfloat16* mW, const float* mB, float* part,
                            double* dW, cudaStream_t st)
{
    const int smem = (int)sizeof(GradSm);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const long long ntile = (R + kGT - 1) / kGT;
    const int G = (int)std::max(1LL, std::min(ntile, (long long)kMaxGradBlocks));
    k_mlp_grad<<<G, kGNT, smem, st>>>(rows, R, mW, mB, part);
    k_mlp_grad_reduce<<<(kMlpNW + 255) / 256, 256, 0, st>>>(part, G, dW);
    return cudaGetLastError();
}

}  // namespace pbe
