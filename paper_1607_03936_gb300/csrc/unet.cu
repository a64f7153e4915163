// Learned pressure-Poisson correction: a 3-level 3-D convolutional U-Net trained and run on the
// GPU with BF16 tensor-core kernels (mma.sync m16n8k16, FP32 accumulation), FP32 master weights
// and Adam.  Architecture (channels 16/32/64, 3x3x3 kernels, average pooling, nearest
// upsampling, skip concatenation, ReLU, linear output) and parameter layout as in wbfbt.h.
//
// Convolutions are implicit GEMMs: M = voxels (16-voxel tiles along x), N = output channels
// (8-wide tiles), K = 27 taps x input channels (16-wide chunks).  Forward and backward-data run
// the same kernel (backward-data with tap-flipped, channel-transposed weights and the ReLU
// mask of the layer input fused into the epilogue); the weight gradient is a second
// tensor-core kernel with the voxel sum split over the warps of a block and reduced in a fixed
// order, so every result is reproducible.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "common.cuh"
#include "unet.h"
#include "wbfbt.h"

namespace {

typedef __nv_bfloat16 bf16;

inline int r16(int c) { return (c + 15) / 16 * 16; }
inline int r8(int c) { return (c + 7) / 8 * 8; }
inline unsigned nb(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__device__ inline void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ inline unsigned ld_pair(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }

__device__ inline unsigned pack2(bf16 lo, bf16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// Neighbour voxel (same sample) of local voxel v at tap t, or -1 outside the grid.
__device__ inline int nbr(int v, int n, int t) {
  const int x = v % n, y = (v / n) % n, z = v / (n * n);
  const int xx = x + t % 3 - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;
  if (xx < 0 || yy < 0 || zz < 0 || xx >= n || yy >= n || zz >= n) return -1;
  return xx + n * (yy + n * zz);
}

// y[b][v][co] = epilogue(sum_t sum_ci W[t][co][ci] x[b][nbr(v,t)][ci]).  One warp per 16-voxel
// tile and NTW of the NT 8-wide output tiles (NTW = NT on large grids; NTW = 1 spreads the output
// tiles over NT warps where voxel tiles are few).  Epilogue: + bias, ReLU, or x mask[v][co] > 0
// (backward data).
template <int NT, int NTW>
__global__ void __launch_bounds__(128) k_conv(int n, int batch, const bf16* __restrict__ x, int ldx, int kp,
                                              const bf16* __restrict__ W, const float* __restrict__ bias, int relu,
                                              const bf16* __restrict__ mask, int ldm, int cvalid,
                                              bf16* __restrict__ y, int ldy, float* __restrict__ yf, int ldyf) {
  pdl_entry();
  constexpr int NG = NT / NTW;
  const int V = n * n * n;
  const int tiles = (V + 15) / 16;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= tiles * batch * NG) return;
  const int grp = gw % NG, warp = gw / NG;
  const int b = warp / tiles, m0 = (warp % tiles) * 16;
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const bf16* xb = x + (size_t)b * V * ldx;
  const int v0 = m0 + gid, v1 = m0 + gid + 8;
  // voxel coordinates once; per tap the neighbour is an offset with a bounds check
  const int x0 = v0 % n, y0 = (v0 / n) % n, z0 = v0 / (n * n);
  const int x1 = v1 % n, y1 = (v1 / n) % n, z1 = v1 / (n * n);
  float acc[NTW][4];
#pragma unroll
  for (int t = 0; t < NTW; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
  for (int tap = 0; tap < 27; ++tap) {
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    const int off = dx + n * (dy + n * dz);
    const bool in0 = v0 < V && (unsigned)(x0 + dx) < (unsigned)n && (unsigned)(y0 + dy) < (unsigned)n &&
                     (unsigned)(z0 + dz) < (unsigned)n;
    const bool in1 = v1 < V && (unsigned)(x1 + dx) < (unsigned)n && (unsigned)(y1 + dy) < (unsigned)n &&
                     (unsigned)(z1 + dz) < (unsigned)n;
    const int n0 = in0 ? v0 + off : -1;
    const int n1 = in1 ? v1 + off : -1;
    const bf16* r0 = xb + (size_t)(n0 < 0 ? 0 : n0) * ldx;
    const bf16* r1 = xb + (size_t)(n1 < 0 ? 0 : n1) * ldx;
    const bf16* wt = W + (size_t)tap * NT * 8 * kp;
    for (int kc = 0; kc < kp; kc += 16) {
      unsigned a[4];
      a[0] = n0 >= 0 ? ld_pair(r0 + kc + tig * 2) : 0u;
      a[1] = n1 >= 0 ? ld_pair(r1 + kc + tig * 2) : 0u;
      a[2] = n0 >= 0 ? ld_pair(r0 + kc + 8 + tig * 2) : 0u;
      a[3] = n1 >= 0 ? ld_pair(r1 + kc + 8 + tig * 2) : 0u;
#pragma unroll
      for (int t = 0; t < NTW; ++t) {
        const bf16* wr = wt + (size_t)((grp * NTW + t) * 8 + gid) * kp + kc;
        unsigned bb[2] = {ld_pair(wr + tig * 2), ld_pair(wr + 8 + tig * 2)};
        mma_bf16(acc[t], a, bb);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NTW; ++t) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = h ? v1 : v0;
      if (v >= V) continue;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int co = (grp * NTW + t) * 8 + tig * 2 + e;
        if (co >= cvalid) continue;
        float val = acc[t][h * 2 + e];
        if (bias) val += bias[co];
        if (relu) val = fmaxf(val, 0.f);
        if (mask && !(__bfloat162float(mask[((size_t)b * V + v) * ldm + co]) > 0.f)) val = 0.f;
        if (y) y[((size_t)b * V + v) * ldy + co] = __float2bfloat16(val);
        if (yf) yf[((size_t)b * V + v) * ldyf + co] = val;
      }
    }
  }
}

// ------------------------------------------------------------------ tcgen05 form of the convolution
// The same implicit GEMM on the fifth-generation tensor cores: a CTA owns 128 consecutive voxels
// of one sample (M = 128) and all NPAD output channels (N = NPAD, a multiple of 16); the K loop
// runs over the 27 taps x 16-channel chunks.  Each chunk's operands are staged in shared memory
// in the canonical no-swizzle K-major layout (8 x 16-byte core matrices: [rows / 8][2][8][16 B],
// so the leading-dimension offset, between the two K halves, is 128 B and the stride offset,
// between 8-row groups, 256 B): A = the 128 voxels' neighbour rows at the tap (zero outside the
// grid), B = the tap's NPAD x 16 weight block.  One thread issues tcgen05.mma (kind::f16, BF16
// inputs, FP32 accumulator in tensor memory) and commits it to the stage's mbarrier; a ring of
// TC_STAGES stages lets the threads fill the next chunks while earlier MMAs run.  The epilogue
// reads the accumulator with tcgen05.ld (warp w: TMEM lanes 32w..32w+31 = voxels) and applies bias,
// ReLU or the backward mask like k_conv.  Waits are bounded: on a timeout the CTA sets
// g_tc_timeout, writes NaN and still frees its tensor memory.

constexpr int TC_STAGES = 4;
constexpr int TC_M = 128;

__device__ int g_tc_timeout;   // set when a tensor-core convolution gave up waiting on its MMAs

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;   // leading-dimension byte offset: the two 8-element K halves
  d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset: consecutive 8-row groups
  d |= (uint64_t)1 << 46;            // descriptor version; base offset 0, no swizzle
  return d;
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
  return done != 0;
}

// One stage = the three x-taps (dx = -1, 0, 1) of one (dy, dz) pair for one 16-channel chunk: three
// A blocks (128 x 16) and three B blocks (NPAD x 16), three MMAs, one commit.  256 threads: two per
// voxel row (one 16-byte half each), so a stage is three 16-byte gathers per thread.
constexpr int TC_THREADS = 256;
constexpr int TC_TAPS = 3;

template <int NPAD>
__host__ __device__ constexpr int tc_stage_bytes() {
  return TC_TAPS * (TC_M * 16 + NPAD * 16) * 2;
}

template <int NPAD>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(int n, int batch, const bf16* __restrict__ x, int ldx, int kp,
                                                       const bf16* __restrict__ W, const float* __restrict__ bias,
                                                       int relu, const bf16* __restrict__ mask, int ldm, int cvalid,
                                                       bf16* __restrict__ y, int ldy, float* __restrict__ yf,
                                                       int ldyf) {
  static_assert(NPAD % 16 == 0 && NPAD >= 16 && NPAD <= 128, "N must be a multiple of 16 in [16, 128]");
  constexpr int TCOLS = NPAD <= 32 ? 32 : (NPAD <= 64 ? 64 : 128);
  constexpr int ABYTES = TC_M * 16 * 2, BBYTES = NPAD * 16 * 2;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[TC_STAGES];
  __shared__ uint32_t tmem_base;
  pdl_entry();
  const int V = n * n * n;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tiles = V / TC_M;
  const int b = blockIdx.x / tiles, v0 = (blockIdx.x % tiles) * TC_M;
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NPAD >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  const int m = tid >> 1, half = tid & 1;           // voxel row and 16-byte half this thread stages
  const int v = v0 + m;
  const int vx = v % n, vy = (v / n) % n, vz = v / (n * n);
  const bf16* xb = x + (size_t)b * V * ldx;
  const int kch = kp / 16, nstages = 9 * kch;       // (dy, dz) pairs x channel chunks
  const int slot = ((m >> 3) * 2 + half) * 8 + (m & 7);   // uint4 index in an A block
  bool ok = true;
  for (int c = 0; c < nstages; ++c) {
    const int s = c % TC_STAGES;
    if (c >= TC_STAGES && ok) ok = tc_wait(smem_addr(&mbar[s]), ((c / TC_STAGES) - 1) & 1);
    const int pair = c / kch, kc = (c % kch) * 16;
    const int dy = pair % 3 - 1, dz = pair / 3 - 1;
    unsigned char* st = tc_smem + (size_t)s * tc_stage_bytes<NPAD>();
    const bool iny = (unsigned)(vy + dy) < (unsigned)n && (unsigned)(vz + dz) < (unsigned)n;
#pragma unroll
    for (int t = 0; t < TC_TAPS; ++t) {
      const int dx = t - 1;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (iny && (unsigned)(vx + dx) < (unsigned)n)
        val = reinterpret_cast<const uint4*>(xb + (size_t)(v + dx + n * (dy + n * dz)) * ldx + kc)[half];
      reinterpret_cast<uint4*>(st + t * ABYTES)[slot] = val;
    }
    for (int q = tid; q < TC_TAPS * NPAD * 2; q += TC_THREADS) {
      const int t = q / (NPAD * 2), r = (q >> 1) % NPAD, hf = q & 1;
      const int tap = t + 3 * (dy + 1) + 9 * (dz + 1);
      const uint4 w = reinterpret_cast<const uint4*>(W + ((size_t)tap * NPAD + r) * kp + kc)[hf];
      reinterpret_cast<uint4*>(st + TC_TAPS * ABYTES + t * BBYTES)[((r >> 3) * 2 + hf) * 8 + (r & 7)] = w;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int t = 0; t < TC_TAPS; ++t) {
        const uint64_t da = tc_smem_desc(smem_addr(st + t * ABYTES));
        const uint64_t db = tc_smem_desc(smem_addr(st + TC_TAPS * ABYTES + t * BBYTES));
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tbase),
            "l"(da), "l"(db), "r"(idesc), "r"((c > 0 || t > 0) ? 1 : 0));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&mbar[s])));
    }
  }
  {
    const int cl = nstages - 1;
    if (ok) ok = tc_wait(smem_addr(&mbar[cl % TC_STAGES]), (cl / TC_STAGES) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok && tid == 0) atomicExch(&g_tc_timeout, 1);
  // epilogue: warps 0-3 read TMEM lanes 32w..32w+31 (voxels), all columns; warps 4-7 idle
  if (warp < 4) {
    const int vv = v0 + warp * 32 + (tid & 31);
    const size_t row = (size_t)b * V + vv;
#pragma unroll
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int co = c0 + j;
        if (co >= cvalid) continue;
        float val = ok ? __uint_as_float(r[j]) : __int_as_float(0x7fc00000);
        if (bias) val += bias[co];
        if (relu) val = fmaxf(val, 0.f);
        if (mask && !(__bfloat162float(mask[row * ldm + co]) > 0.f)) val = 0.f;
        if (y) y[row * ldy + co] = __float2bfloat16(val);
        if (yf) yf[row * ldyf + co] = val;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS));
}

// dW[t][ci][co] = sum_{b,v} x[b][nbr(v,t)][ci] g[b][v][co]: block per (tap, 16-channel ci tile),
// 8 warps split the voxels, partial tiles reduced in warp order.  With gridDim.z = S > 1 the
// voxel chunks are also split over S blocks (chunk kk goes to block kk / 8 mod S), each block
// writing its partial tile to part[blockIdx.z]; k_wgrad_sum adds the S partials in order.
template <int NT>
__global__ void __launch_bounds__(256) k_wgrad(int n, int batch, const bf16* __restrict__ x, int ldx, int cin,
                                               const bf16* __restrict__ g, int ldg, int cout,
                                               float* __restrict__ dW, float* __restrict__ part) {
  pdl_entry();
  const int V = n * n * n, tot = V * batch;
  const int tap = blockIdx.x, ci0 = blockIdx.y * 16;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
  const int ks = (tot + 15) / 16;
  const int S = gridDim.z;
  float* out = S > 1 ? part + (size_t)blockIdx.z * 27 * cin * cout : dW;
  for (int kk = blockIdx.z * 8 + w; kk < ks; kk += 8 * S) {
    const int k0 = kk * 16;
    // A: 16 (ci) x 16 (voxels); B: 16 (voxels) x 8 (co)
    bf16 xa[4][2];
    int vk[4];
    const int kidx[4] = {k0 + tig * 2, k0 + tig * 2 + 1, k0 + tig * 2 + 8, k0 + tig * 2 + 9};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gv = kidx[q];
      vk[q] = gv < tot ? gv : -1;
    }
    unsigned a[4];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {     // rows gid (hh=0) and gid+8 (hh=1)
      const int ci = ci0 + gid + hh * 8;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bf16 val = __float2bfloat16(0.f);
        if (vk[q] >= 0 && ci < cin) {
          const int bb = vk[q] / V, v = vk[q] % V;
          const int nv = nbr(v, n, tap);
          if (nv >= 0) val = x[((size_t)bb * V + nv) * ldx + ci];
        }
        xa[q][hh] = val;
      }
    }
    a[0] = pack2(xa[0][0], xa[1][0]);
    a[1] = pack2(xa[0][1], xa[1][1]);
    a[2] = pack2(xa[2][0], xa[3][0]);
    a[3] = pack2(xa[2][1], xa[3][1]);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int co = t * 8 + gid;
      bf16 gb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        gb[q] = (vk[q] >= 0 && co < cout) ? g[(size_t)vk[q] * ldg + co] : __float2bfloat16(0.f);
      unsigned bb[2] = {pack2(gb[0], gb[1]), pack2(gb[2], gb[3])};
      mma_bf16(acc[t], a, bb);
    }
  }
  __shared__ float red[8][16][NT * 8];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    red[w][gid][t * 8 + tig * 2] = acc[t][0];
    red[w][gid][t * 8 + tig * 2 + 1] = acc[t][1];
    red[w][gid + 8][t * 8 + tig * 2] = acc[t][2];
    red[w][gid + 8][t * 8 + tig * 2 + 1] = acc[t][3];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 16 * NT * 8; idx += blockDim.x) {
    const int r = idx / (NT * 8), c = idx % (NT * 8);
    float s = 0.f;
    for (int ww = 0; ww < 8; ++ww) s += red[ww][r][c];
    const int ci = ci0 + r;
    if (ci < cin && c < cout) out[((size_t)tap * cin + ci) * cout + c] = s;
  }
}

// dW[i] = sum_{s < S} part[s][i], in the order of s (reproducible).
__global__ void k_wgrad_sum(int S, long long n, const float* __restrict__ part, float* __restrict__ dW) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.f;
  for (int s2 = 0; s2 < S; ++s2) acc += part[(size_t)s2 * n + i];
  dW[i] = acc;
}

// db[co] = sum over rows of g[row][co] (one block per channel, fixed tree)
__global__ void k_colsum(const bf16* __restrict__ g, int ldg, long long rows, float* __restrict__ db) {
  pdl_entry();
  const int co = blockIdx.x;
  float s = 0.f;
  for (long long r = threadIdx.x; r < rows; r += blockDim.x) s += __bfloat162float(g[r * ldg + co]);
  __shared__ float sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[co] = sh[0];
}

// 2x2x2 average pooling: out [b][n/2 grid][c] from in [b][n grid][c]
__global__ void k_pool(int n, int batch, int c, const bf16* __restrict__ in, int ldi, bf16* __restrict__ out,
                       int ldo) {
  pdl_entry();
  const int m = n / 2, Vo = m * m * m;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)Vo * batch * c) return;
  const int ch = (int)(t % c);
  const long long vv = t / c;
  const int b = (int)(vv / Vo), v = (int)(vv % Vo);
  const int x = v % m, y = (v / m) % m, z = v / (m * m);
  float s = 0.f;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int vi = (2 * x + dx) + n * ((2 * y + dy) + n * (2 * z + dz));
        s += __bfloat162float(in[((size_t)b * n * n * n + vi) * ldi + ch]);
      }
  out[((size_t)b * Vo + v) * ldo + ch] = __float2bfloat16(s * 0.125f);
}

// nearest upsampling: out [b][2m grid][c] (channel slice) from in [b][m grid][c]
__global__ void k_upsample(int m, int batch, int c, const bf16* __restrict__ in, int ldi, bf16* __restrict__ out,
                           int ldo) {
  pdl_entry();
  const int n = 2 * m, V = n * n * n;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)V * batch * c) return;
  const int ch = (int)(t % c);
  const long long vv = t / c;
  const int b = (int)(vv / V), v = (int)(vv % V);
  const int x = v % n, y = (v / n) % n, z = v / (n * n);
  const int vp = (x / 2) + m * ((y / 2) + m * (z / 2));
  out[((size_t)b * V + v) * ldo + ch] = in[((size_t)b * m * m * m + vp) * ldi + ch];
}

// g_out[b][vp][c] = sum over the 8 children of g_in (backward of nearest upsampling)
__global__ void k_upsample_bwd(int m, int batch, int c, const bf16* __restrict__ gin, int ldi, bf16* __restrict__ gout,
                               int ldo) {
  pdl_entry();
  const int n = 2 * m, Vp = m * m * m;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)Vp * batch * c) return;
  const int ch = (int)(t % c);
  const long long vv = t / c;
  const int b = (int)(vv / Vp), v = (int)(vv % Vp);
  const int x = v % m, y = (v / m) % m, z = v / (m * m);
  float s = 0.f;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int vi = (2 * x + dx) + n * ((2 * y + dy) + n * (2 * z + dz));
        s += __bfloat162float(gin[((size_t)b * n * n * n + vi) * ldi + ch]);
      }
  gout[((size_t)b * Vp + v) * ldo + ch] = __float2bfloat16(s);
}

// g[b][v][c] = skip[b][v][c] + (act[b][v][c] > 0 ? gp[b][parent(v)][c] / 8 : 0)
// (skip already carries the ReLU mask; the pooled path takes it here)
__global__ void k_skip_pool_bwd(int n, int batch, int c, const bf16* __restrict__ skip, int lds,
                                const bf16* __restrict__ act, int lda, const bf16* __restrict__ gp, int ldp,
                                bf16* __restrict__ g, int ldg) {
  pdl_entry();
  const int V = n * n * n, m = n / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)V * batch * c) return;
  const int ch = (int)(t % c);
  const long long vv = t / c;
  const int b = (int)(vv / V), v = (int)(vv % V);
  const int x = v % n, y = (v / n) % n, z = v / (n * n);
  const int vp = (x / 2) + m * ((y / 2) + m * (z / 2));
  float s = __bfloat162float(skip[((size_t)b * V + v) * lds + ch]);
  if (__bfloat162float(act[((size_t)b * V + v) * lda + ch]) > 0.f)
    s += 0.125f * __bfloat162float(gp[((size_t)b * m * m * m + vp) * ldp + ch]);
  g[((size_t)b * V + v) * ldg + ch] = __float2bfloat16(s);
}

// input FP32 [rows][cin] -> BF16 [rows][ld] (padding zero)
__global__ void k_pack_input(long long rows, int cin, int ld, const float* __restrict__ x, bf16* __restrict__ out) {
  pdl_entry();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * ld) return;
  const long long r = t / ld;
  const int c = (int)(t % ld);
  out[t] = __float2bfloat16(c < cin ? x[r * cin + c] : 0.f);
}

// MSE: diff = y - target; per-block partial sums of squares; gradient 2 diff / count in BF16 [rows][ld]
__global__ void k_mse(long long rows, int cout, const float* __restrict__ y, const float* __restrict__ tgt, int ld,
                      double inv_count, bf16* __restrict__ g, double* __restrict__ part) {
  pdl_entry();
  double s = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < rows * ld;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / ld;
    const int c = (int)(t % ld);
    float gv = 0.f;
    if (c < cout) {
      const double d = (double)y[r * cout + c] - (double)tgt[r * cout + c];
      s += d * d;
      gv = (float)(2.0 * d * inv_count);
    }
    g[t] = __float2bfloat16(gv);
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_parts(int np, const double* __restrict__ part, double scale, double* __restrict__ out) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    out[0] = s * scale;
  }
}

__global__ void k_adam(long long n, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 kernel weights from the FP32 master W[t][ci][co]:
//   Wt[t][co][ci]  (np8 x kp16, forward)     Wf[t][ci][co] = W[26 - t][ci][co] (npb8 x kpb16, backward data)
__global__ void k_refresh_weights(int cin, int cout, const float* __restrict__ W, int kp, int npf, bf16* __restrict__ Wt,
                                  int kpb, int npb, bf16* __restrict__ Wf) {
  pdl_entry();
  const int tap = blockIdx.x;
  for (int idx = threadIdx.x; idx < npf * kp; idx += blockDim.x) {
    const int co = idx / kp, ci = idx % kp;
    const float v = (co < cout && ci < cin) ? W[((size_t)tap * cin + ci) * cout + co] : 0.f;
    Wt[(size_t)tap * npf * kp + idx] = __float2bfloat16(v);
  }
  for (int idx = threadIdx.x; idx < npb * kpb; idx += blockDim.x) {
    const int ci = idx / kpb, co = idx % kpb;
    const float v = (co < cout && ci < cin) ? W[((size_t)(26 - tap) * cin + ci) * cout + co] : 0.f;
    Wf[(size_t)tap * npb * kpb + idx] = __float2bfloat16(v);
  }
}

struct Layer {
  int cin, cout, kp, npf, kpb, npb;
  size_t woff, boff;   // offsets into the flat parameter vector
  bf16 *Wt = nullptr, *Wf = nullptr;
};

template <int NT>
void conv_launch(int n, int batch, const bf16* x, int ldx, int kp, const bf16* W, const float* bias, int relu,
                 const bf16* mask, int ldm, int cvalid, bf16* y, int ldy, float* yf, int ldyf, cudaStream_t st) {
  const long long warps = (long long)((n * n * n + 15) / 16) * batch;
  if (warps >= 152 * 8)   // enough voxel tiles to fill the GPU: one warp per tile, all output tiles
    wb_launch(k_conv<NT, NT>, nb(warps * 32, 128), 128, 0, st, n, batch, x, ldx, kp, W, bias, relu, mask, ldm,
              cvalid, y, ldy, yf, ldyf);
  else                    // few voxel tiles: one warp per (tile, 8-channel output tile)
    wb_launch(k_conv<NT, 1>, nb(warps * NT * 32, 128), 128, 0, st, n, batch, x, ldx, kp, W, bias, relu, mask, ldm,
              cvalid, y, ldy, yf, ldyf);
}

template <int NPAD>
void conv_tc_launch(int n, int batch, const bf16* x, int ldx, int kp, const bf16* W, const float* bias, int relu,
                    const bf16* mask, int ldm, int cvalid, bf16* y, int ldy, float* yf, int ldyf, cudaStream_t st) {
  constexpr size_t smem = (size_t)TC_STAGES * tc_stage_bytes<NPAD>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv_tc<NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const unsigned blocks = (unsigned)((long long)n * n * n / TC_M * batch);
  wb_launch(k_conv_tc<NPAD>, blocks, TC_THREADS, smem, st, n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y,
            ldy, yf, ldyf);
}

// Layers with a multiple of 16 padded output channels on grids of at least 152 tiles of 128 voxels
// (one CTA per tile: enough to fill the SMs) run on the tcgen05 kernel; the others (the coarser
// levels, which have few tiles, and the 4- and 8-channel layers) on the mma.sync one, which
// spreads the output-channel tiles over warps.  Measured at 32^3: the 16-channel layers 19.4 us on
// tcgen05 against 21 us; on 16^3 (32 tiles) 30.6 against 26 us, on 8^3 (4 tiles) 52 against 28 us.
void conv(int npad, int n, int batch, const bf16* x, int ldx, int kp, const bf16* W, const float* bias, int relu,
          const bf16* mask, int ldm, int cvalid, bf16* y, int ldy, float* yf, int ldyf, cudaStream_t st) {
  const long long vox = (long long)n * n * n;
  if (vox % TC_M == 0 && kp % 16 == 0 && vox / TC_M * batch >= 152) {
    switch (npad) {
      case 16: conv_tc_launch<16>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); return;
      case 32: conv_tc_launch<32>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); return;
      case 48: conv_tc_launch<48>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); return;
      case 64: conv_tc_launch<64>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); return;
      case 96: conv_tc_launch<96>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); return;
      default: break;
    }
  }
  switch (npad / 8) {
    case 1: conv_launch<1>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); break;
    case 2: conv_launch<2>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); break;
    case 4: conv_launch<4>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); break;
    case 6: conv_launch<6>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); break;
    case 8: conv_launch<8>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); break;
    case 12: conv_launch<12>(n, batch, x, ldx, kp, W, bias, relu, mask, ldm, cvalid, y, ldy, yf, ldyf, st); break;
    default: break;
  }
}

constexpr int WGRAD_MAX_SPLIT = 8;

// Blocks in z (voxel-chunk split) for a weight gradient: fill about two blocks per SM, keep at
// least four 16-voxel chunks per warp, at most WGRAD_MAX_SPLIT.
int wgrad_split(int n, int batch, int cin) {
  const long long ks = ((long long)n * n * n * batch + 15) / 16;
  const int tiles = 27 * ((cin + 15) / 16);
  int S = (2 * 152 + tiles - 1) / tiles;
  while (S > 1 && ks < 8LL * 4 * S) --S;
  return std::max(1, std::min(S, WGRAD_MAX_SPLIT));
}

void wgrad(int n, int batch, const bf16* x, int ldx, int cin, const bf16* g, int ldg, int cout, float* dW,
           float* part, cudaStream_t st) {
  const int S = part ? wgrad_split(n, batch, cin) : 1;
  dim3 grid(27, (cin + 15) / 16, S);
  switch (r8(cout) / 8) {
    case 1: wb_launch(k_wgrad<1>, grid, 256, 0, st, n, batch, x, ldx, cin, g, ldg, cout, dW, part); break;
    case 2: wb_launch(k_wgrad<2>, grid, 256, 0, st, n, batch, x, ldx, cin, g, ldg, cout, dW, part); break;
    case 4: wb_launch(k_wgrad<4>, grid, 256, 0, st, n, batch, x, ldx, cin, g, ldg, cout, dW, part); break;
    case 8: wb_launch(k_wgrad<8>, grid, 256, 0, st, n, batch, x, ldx, cin, g, ldg, cout, dW, part); break;
    default: break;
  }
  if (S > 1) {
    const long long cnt = 27LL * cin * cout;
    wb_launch(k_wgrad_sum, nb(cnt, 256), 256, 0, st, S, cnt, (const float*)part, dW);
  }
}

}  // namespace

struct wbfbt_net {
  cudaStream_t st = nullptr;
  int cin = 0, cout = 0, n = 0, max_batch = 0;
  long long nparam = 0;
  std::vector<Layer> L;
  std::vector<void*> allocs;
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  float* wpart = nullptr;   // split weight-gradient partials [WGRAD_MAX_SPLIT][largest 27 cin cout]
  double *part = nullptr, *dloss = nullptr;
  int adam_t = 0;
  // activations (BF16, [batch][voxels][ld])
  bf16 *x0, *a1, *cat2, *p2, *a3, *cat1, *p4, *a5, *a6, *a7, *a8, *a9, *a10;
  float* yout;   // [batch][V0][cout]
  // gradients
  bf16 *g11, *g10, *g9, *gcat2, *g8, *g7, *gcat1, *g6, *g5, *gp4, *g4, *g3, *gp2, *g2, *g1;
  template <typename T>
  T* get(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, (n ? n : 1) * sizeof(T)) != cudaSuccess) throw 1;
    allocs.push_back(p);
    return static_cast<T*>(p);
  }
  ~wbfbt_net() {
    if (st) cudaStreamSynchronize(st);
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

const int kLayerCin[11] = {-1, 16, 16, 32, 32, 64, 96, 32, 48, 16, 16};
const int kLayerCout[11] = {16, 16, 32, 32, 64, 64, 32, 32, 16, 16, -1};

void refresh_all(wbfbt_net* net) {
  for (auto& l : net->L)
    wb_launch(k_refresh_weights, 27, 256, 0, net->st, l.cin, l.cout, net->theta + l.woff, l.kp, l.npf, l.Wt,
                                                                   l.kpb, l.npb, l.Wf);
}

void forward(wbfbt_net* N, const float* x, int B) {
  const cudaStream_t st = N->st;
  const int n0 = N->n, n1 = n0 / 2, n2 = n0 / 4;
  const long long V0 = (long long)n0 * n0 * n0;
  auto& L = N->L;
  auto bias = [&](int i) { return N->theta + L[i].boff; };
  wb_launch(k_pack_input, nb(V0 * B * 16, 256), 256, 0, st, V0 * B, N->cin, 16, x, N->x0);
  conv(L[0].npf, n0, B, N->x0, 16, L[0].kp, L[0].Wt, bias(0), 1, nullptr, 0, 16, N->a1, 16, nullptr, 0, st);
  conv(L[1].npf, n0, B, N->a1, 16, L[1].kp, L[1].Wt, bias(1), 1, nullptr, 0, 16, N->cat2 + 32, 48, nullptr, 0, st);
  wb_launch(k_pool, nb((long long)n1 * n1 * n1 * B * 16, 256), 256, 0, st, n0, B, 16, N->cat2 + 32, 48, N->p2, 16);
  conv(L[2].npf, n1, B, N->p2, 16, L[2].kp, L[2].Wt, bias(2), 1, nullptr, 0, 32, N->a3, 32, nullptr, 0, st);
  conv(L[3].npf, n1, B, N->a3, 32, L[3].kp, L[3].Wt, bias(3), 1, nullptr, 0, 32, N->cat1 + 64, 96, nullptr, 0, st);
  wb_launch(k_pool, nb((long long)n2 * n2 * n2 * B * 32, 256), 256, 0, st, n1, B, 32, N->cat1 + 64, 96, N->p4, 32);
  conv(L[4].npf, n2, B, N->p4, 32, L[4].kp, L[4].Wt, bias(4), 1, nullptr, 0, 64, N->a5, 64, nullptr, 0, st);
  conv(L[5].npf, n2, B, N->a5, 64, L[5].kp, L[5].Wt, bias(5), 1, nullptr, 0, 64, N->a6, 64, nullptr, 0, st);
  wb_launch(k_upsample, nb((long long)n1 * n1 * n1 * B * 64, 256), 256, 0, st, n2, B, 64, N->a6, 64, N->cat1, 96);
  conv(L[6].npf, n1, B, N->cat1, 96, L[6].kp, L[6].Wt, bias(6), 1, nullptr, 0, 32, N->a7, 32, nullptr, 0, st);
  conv(L[7].npf, n1, B, N->a7, 32, L[7].kp, L[7].Wt, bias(7), 1, nullptr, 0, 32, N->a8, 32, nullptr, 0, st);
  wb_launch(k_upsample, nb(V0 * B * 32, 256), 256, 0, st, n1, B, 32, N->a8, 32, N->cat2, 48);
  conv(L[8].npf, n0, B, N->cat2, 48, L[8].kp, L[8].Wt, bias(8), 1, nullptr, 0, 16, N->a9, 16, nullptr, 0, st);
  conv(L[9].npf, n0, B, N->a9, 16, L[9].kp, L[9].Wt, bias(9), 1, nullptr, 0, 16, N->a10, 16, nullptr, 0, st);
  conv(L[10].npf, n0, B, N->a10, 16, L[10].kp, L[10].Wt, bias(10), 0, nullptr, 0, N->cout, nullptr, 0, N->yout,
       N->cout, st);
}

void backward(wbfbt_net* N, int B) {
  const cudaStream_t st = N->st;
  const int n0 = N->n, n1 = n0 / 2, n2 = n0 / 4;
  const long long V0 = (long long)n0 * n0 * n0, V1 = (long long)n1 * n1 * n1, V2 = (long long)n2 * n2 * n2;
  auto& L = N->L;
  float* G = N->grad;
  auto layer_grads = [&](int i, int n, const bf16* xin, int ldx, const bf16* g, int ldg, long long rows) {
    wgrad(n, B, xin, ldx, L[i].cin, g, ldg, L[i].cout, G + L[i].woff, N->wpart, st);
    wb_launch(k_colsum, L[i].cout, 256, 0, st, g, ldg, rows, G + L[i].boff);
  };
  // bwd data: input g (ld kpb), output (ld of the layer input), ReLU mask of the layer input
  auto bwd = [&](int i, int n, const bf16* g, const bf16* mask, int ldm, bf16* out, int ldo) {
    conv(L[i].npb, n, B, g, L[i].kpb, L[i].kpb, L[i].Wf, nullptr, 0, mask, ldm, L[i].cin, out, ldo, nullptr, 0, st);
  };
  layer_grads(10, n0, N->a10, 16, N->g11, 16, V0 * B);
  bwd(10, n0, N->g11, N->a10, 16, N->g10, 16);
  layer_grads(9, n0, N->a9, 16, N->g10, 16, V0 * B);
  bwd(9, n0, N->g10, N->a9, 16, N->g9, 16);
  layer_grads(8, n0, N->cat2, 48, N->g9, 16, V0 * B);
  bwd(8, n0, N->g9, N->cat2, 48, N->gcat2, 48);
  wb_launch(k_upsample_bwd, nb(V1 * B * 32, 256), 256, 0, st, n1, B, 32, N->gcat2, 48, N->g8, 32);
  layer_grads(7, n1, N->a7, 32, N->g8, 32, V1 * B);
  bwd(7, n1, N->g8, N->a7, 32, N->g7, 32);
  layer_grads(6, n1, N->cat1, 96, N->g7, 32, V1 * B);
  bwd(6, n1, N->g7, N->cat1, 96, N->gcat1, 96);
  wb_launch(k_upsample_bwd, nb(V2 * B * 64, 256), 256, 0, st, n2, B, 64, N->gcat1, 96, N->g6, 64);
  layer_grads(5, n2, N->a5, 64, N->g6, 64, V2 * B);
  bwd(5, n2, N->g6, N->a5, 64, N->g5, 64);
  layer_grads(4, n2, N->p4, 32, N->g5, 64, V2 * B);
  bwd(4, n2, N->g5, nullptr, 0, N->gp4, 32);
  wb_launch(k_skip_pool_bwd, nb(V1 * B * 32, 256), 256, 0, st, n1, B, 32, N->gcat1 + 64, 96, N->cat1 + 64, 96,
                                                                           N->gp4, 32, N->g4, 32);
  layer_grads(3, n1, N->a3, 32, N->g4, 32, V1 * B);
  bwd(3, n1, N->g4, N->a3, 32, N->g3, 32);
  layer_grads(2, n1, N->p2, 16, N->g3, 32, V1 * B);
  bwd(2, n1, N->g3, nullptr, 0, N->gp2, 16);
  wb_launch(k_skip_pool_bwd, nb(V0 * B * 16, 256), 256, 0, st, n0, B, 16, N->gcat2 + 32, 48, N->cat2 + 32, 48,
                                                                           N->gp2, 16, N->g2, 16);
  layer_grads(1, n0, N->a1, 16, N->g2, 16, V0 * B);
  bwd(1, n0, N->g2, N->a1, 16, N->g1, 16);
  layer_grads(0, n0, N->x0, 16, N->g1, 16, V0 * B);
}

template <class F>
int net_guard(wbfbt_net* N, F f) {
  try {
    f();
    return cudaGetLastError() == cudaSuccess ? WBFBT_OK : WBFBT_ERR_CUDA;
  } catch (...) {
    return WBFBT_ERR_CUDA;
  }
}

}  // namespace

extern "C" {

long long wbfbt_net_num_params(int cin, int cout) {
  long long s = 0;
  for (int i = 0; i < 11; ++i) {
    const long long ci = kLayerCin[i] < 0 ? cin : kLayerCin[i], co = kLayerCout[i] < 0 ? cout : kLayerCout[i];
    s += 27 * ci * co + co;
  }
  return s;
}

int wbfbt_net_create(int cin, int cout, int n, int max_batch, void* stream, wbfbt_net** out) {
  if (!out || cin < 1 || cin > 16 || cout < 1 || cout > 16 || n < 4 || n % 4 != 0 || max_batch < 1)
    return WBFBT_ERR_INVALID;
  *out = nullptr;
  auto N = std::make_unique<wbfbt_net>();
  N->st = (cudaStream_t)stream;
  N->cin = cin;
  N->cout = cout;
  N->n = n;
  N->max_batch = max_batch;
  try {
    size_t off = 0;
    for (int i = 0; i < 11; ++i) {
      Layer l;
      l.cin = kLayerCin[i] < 0 ? cin : kLayerCin[i];
      l.cout = kLayerCout[i] < 0 ? cout : kLayerCout[i];
      l.kp = r16(l.cin);
      l.npf = r8(l.cout);
      l.kpb = r16(l.cout);
      l.npb = r8(l.cin);
      l.woff = off;
      off += (size_t)27 * l.cin * l.cout;
      l.boff = off;
      off += l.cout;
      l.Wt = N->get<bf16>((size_t)27 * l.npf * l.kp);
      l.Wf = N->get<bf16>((size_t)27 * l.npb * l.kpb);
      N->L.push_back(l);
    }
    N->nparam = (long long)off;
    size_t wmax = 0;
    for (const auto& l : N->L) wmax = std::max(wmax, (size_t)27 * l.cin * l.cout);
    N->wpart = N->get<float>((size_t)WGRAD_MAX_SPLIT * wmax);
    N->theta = N->get<float>(off);
    N->grad = N->get<float>(off);
    N->m1 = N->get<float>(off);
    N->m2 = N->get<float>(off);
    cudaMemsetAsync(N->theta, 0, off * sizeof(float), N->st);
    cudaMemsetAsync(N->m1, 0, off * sizeof(float), N->st);
    cudaMemsetAsync(N->m2, 0, off * sizeof(float), N->st);
    N->part = N->get<double>(1024);
    N->dloss = N->get<double>(1);
    const size_t B = max_batch, V0 = (size_t)n * n * n, V1 = V0 / 8, V2 = V1 / 8;
    N->x0 = N->get<bf16>(B * V0 * 16);
    N->a1 = N->get<bf16>(B * V0 * 16);
    N->cat2 = N->get<bf16>(B * V0 * 48);
    N->p2 = N->get<bf16>(B * V1 * 16);
    N->a3 = N->get<bf16>(B * V1 * 32);
    N->cat1 = N->get<bf16>(B * V1 * 96);
    N->p4 = N->get<bf16>(B * V2 * 32);
    N->a5 = N->get<bf16>(B * V2 * 64);
    N->a6 = N->get<bf16>(B * V2 * 64);
    N->a7 = N->get<bf16>(B * V1 * 32);
    N->a8 = N->get<bf16>(B * V1 * 32);
    N->a9 = N->get<bf16>(B * V0 * 16);
    N->a10 = N->get<bf16>(B * V0 * 16);
    N->yout = N->get<float>(B * V0 * cout);
    N->g11 = N->get<bf16>(B * V0 * 16);
    N->g10 = N->get<bf16>(B * V0 * 16);
    N->g9 = N->get<bf16>(B * V0 * 16);
    N->gcat2 = N->get<bf16>(B * V0 * 48);
    N->g8 = N->get<bf16>(B * V1 * 32);
    N->g7 = N->get<bf16>(B * V1 * 32);
    N->gcat1 = N->get<bf16>(B * V1 * 96);
    N->g6 = N->get<bf16>(B * V2 * 64);
    N->g5 = N->get<bf16>(B * V2 * 64);
    N->gp4 = N->get<bf16>(B * V2 * 32);
    N->g4 = N->get<bf16>(B * V1 * 32);
    N->g3 = N->get<bf16>(B * V1 * 32);
    N->gp2 = N->get<bf16>(B * V1 * 16);
    N->g2 = N->get<bf16>(B * V0 * 16);
    N->g1 = N->get<bf16>(B * V0 * 16);
    refresh_all(N.get());
    if (cudaStreamSynchronize(N->st) != cudaSuccess) return WBFBT_ERR_CUDA;
  } catch (...) {
    return WBFBT_ERR_CUDA;
  }
  *out = N.release();
  return WBFBT_OK;
}

void wbfbt_net_destroy(wbfbt_net* net) { delete net; }

int wbfbt_net_set_params(wbfbt_net* N, const float* theta) {
  if (!N || !theta) return WBFBT_ERR_INVALID;
  return net_guard(N, [&]() {
    if (cudaMemcpyAsync(N->theta, theta, sizeof(float) * N->nparam, cudaMemcpyDefault, N->st) != cudaSuccess) throw 1;
    cudaMemsetAsync(N->m1, 0, sizeof(float) * N->nparam, N->st);
    cudaMemsetAsync(N->m2, 0, sizeof(float) * N->nparam, N->st);
    N->adam_t = 0;
    refresh_all(N);
  });
}

int wbfbt_net_get_params(wbfbt_net* N, float* theta) {
  if (!N || !theta) return WBFBT_ERR_INVALID;
  return net_guard(N, [&]() {
    if (cudaMemcpyAsync(theta, N->theta, sizeof(float) * N->nparam, cudaMemcpyDefault, N->st) != cudaSuccess) throw 1;
    cudaStreamSynchronize(N->st);
  });
}

int wbfbt_net_forward(wbfbt_net* N, const float* x, int batch, float* y) {
  if (!N || !x || !y || batch < 1 || batch > N->max_batch) return WBFBT_ERR_INVALID;
  return net_guard(N, [&]() {
    forward(N, x, batch);
    const size_t cnt = (size_t)batch * N->n * N->n * N->n * N->cout;
    if (cudaMemcpyAsync(y, N->yout, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, N->st) != cudaSuccess) throw 1;
  });
}

int wbfbt_net_loss_grad(wbfbt_net* N, const float* x, const float* target, int batch, double* loss, float* grad) {
  if (!N || !x || !target || batch < 1 || batch > N->max_batch) return WBFBT_ERR_INVALID;
  return net_guard(N, [&]() {
    forward(N, x, batch);
    const long long rows = (long long)batch * N->n * N->n * N->n;
    const double inv = 1.0 / (double)(rows * N->cout);
    const int blocks = 512;
    wb_launch(k_mse, blocks, 256, 0, N->st, rows, N->cout, N->yout, target, 16, inv, N->g11, N->part);
    wb_launch(k_sum_parts, 1, 32, 0, N->st, blocks, N->part, inv, N->dloss);
    backward(N, batch);
    if (grad && cudaMemcpyAsync(grad, N->grad, sizeof(float) * N->nparam, cudaMemcpyDefault, N->st) != cudaSuccess)
      throw 1;
    if (loss) {
      if (cudaMemcpyAsync(loss, N->dloss, sizeof(double), cudaMemcpyDeviceToHost, N->st) != cudaSuccess) throw 1;
      cudaStreamSynchronize(N->st);
    }
  });
}

int wbfbt_net_adam_step(wbfbt_net* N, float lr) {
  if (!N || !(lr > 0.f)) return WBFBT_ERR_INVALID;
  return net_guard(N, [&]() {
    N->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)N->adam_t), c2 = 1.f - powf(b2, (float)N->adam_t);
    wb_launch(k_adam, nb(N->nparam, 256), 256, 0, N->st, N->nparam, N->theta, N->m1, N->m2, N->grad, lr, b1, b2,
                                                                      1e-8f, c1, c2);
    refresh_all(N);
  });
}

long long wbfbt_net_param_count(const wbfbt_net* N) { return N ? N->nparam : 0; }

int wbfbt_net_save(wbfbt_net* N, const char* path) {
  if (!N || !path) return WBFBT_ERR_INVALID;
  std::vector<float> h((size_t)N->nparam * 3);
  if (cudaMemcpyAsync(h.data(), N->theta, sizeof(float) * N->nparam, cudaMemcpyDeviceToHost, N->st) != cudaSuccess ||
      cudaMemcpyAsync(h.data() + N->nparam, N->m1, sizeof(float) * N->nparam, cudaMemcpyDeviceToHost, N->st) != cudaSuccess ||
      cudaMemcpyAsync(h.data() + 2 * N->nparam, N->m2, sizeof(float) * N->nparam, cudaMemcpyDeviceToHost, N->st) !=
          cudaSuccess ||
      cudaStreamSynchronize(N->st) != cudaSuccess)
    return WBFBT_ERR_CUDA;
  FILE* f = fopen(path, "wb");
  if (!f) return WBFBT_ERR_INVALID;
  const int hdr[6] = {0x57424E54, 1, N->cin, N->cout, N->n, N->adam_t};   // "WBNT", version 1
  const long long np = N->nparam;
  bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(&np, sizeof(np), 1, f) == 1 &&
            fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? WBFBT_OK : WBFBT_ERR_INVALID;
}

int wbfbt_net_load(wbfbt_net* N, const char* path) {
  if (!N || !path) return WBFBT_ERR_INVALID;
  FILE* f = fopen(path, "rb");
  if (!f) return WBFBT_ERR_INVALID;
  int hdr[6];
  long long np = 0;
  bool ok = fread(hdr, sizeof(hdr), 1, f) == 1 && fread(&np, sizeof(np), 1, f) == 1 && hdr[0] == 0x57424E54 &&
            hdr[1] == 1 && hdr[2] == N->cin && hdr[3] == N->cout && np == N->nparam;
  std::vector<float> h(ok ? (size_t)np * 3 : 0);
  ok = ok && fread(h.data(), sizeof(float), h.size(), f) == h.size();
  fclose(f);
  if (!ok) return WBFBT_ERR_INVALID;
  N->adam_t = hdr[5];
  if (cudaMemcpyAsync(N->theta, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice, N->st) != cudaSuccess ||
      cudaMemcpyAsync(N->m1, h.data() + np, sizeof(float) * np, cudaMemcpyHostToDevice, N->st) != cudaSuccess ||
      cudaMemcpyAsync(N->m2, h.data() + 2 * np, sizeof(float) * np, cudaMemcpyHostToDevice, N->st) != cudaSuccess)
    return WBFBT_ERR_CUDA;
  refresh_all(N);
  return cudaStreamSynchronize(N->st) == cudaSuccess ? WBFBT_OK : WBFBT_ERR_CUDA;
}

int wbfbt_net_conv_layer(wbfbt_net* N, int layer, int n, int batch, const float* x, float* y, const float* g,
                         float* dW) {
  if (!N || layer < 0 || layer > 10 || n < 1 || n > 1024 || batch < 1 || !x || (!y && !(g && dW)) ||
      ((g == nullptr) != (dW == nullptr)))
    return WBFBT_ERR_INVALID;
  const Layer& l = N->L[layer];
  const long long rows = (long long)n * n * n * batch;
  bf16 *xb = nullptr, *gb = nullptr;
  const int ldg = r16(l.cout);
  int st = WBFBT_OK;
  if (cudaMalloc(&xb, sizeof(bf16) * rows * l.kp) != cudaSuccess) return WBFBT_ERR_CUDA;
  if (g && cudaMalloc(&gb, sizeof(bf16) * rows * ldg) != cudaSuccess) {
    cudaFree(xb);
    return WBFBT_ERR_CUDA;
  }
  st = net_guard(N, [&]() {
    wb_launch(k_pack_input, nb(rows * l.kp, 256), 256, 0, N->st, rows, l.cin, l.kp, x, xb);
    if (y)
      conv(l.npf, n, batch, xb, l.kp, l.kp, l.Wt, N->theta + l.boff, layer < 10 ? 1 : 0, nullptr, 0, l.cout, nullptr,
           0, y, l.cout, N->st);
    if (g) {
      wb_launch(k_pack_input, nb(rows * ldg, 256), 256, 0, N->st, rows, l.cout, ldg, g, gb);
      wgrad(n, batch, xb, l.kp, l.cin, gb, ldg, l.cout, dW, N->wpart, N->st);
    }
    if (cudaStreamSynchronize(N->st) != cudaSuccess) throw 1;
    int timeout = 0;   // a tensor-core convolution that gave up waiting on its MMAs
    if (cudaMemcpyFromSymbol(&timeout, g_tc_timeout, sizeof(int)) != cudaSuccess || timeout) throw 1;
  });
  cudaFree(xb);
  if (gb) cudaFree(gb);
  return st;
}

}  // extern "C"

// Forward for the solver: x [n^3][cin] FP32 device -> y [n^3][cout] FP32 device (batch 1), on st.
int unet_forward_into(wbfbt_net* N, const float* x, float* y, cudaStream_t st) {
  const cudaStream_t keep = N->st;
  N->st = st;
  int r = net_guard(N, [&]() {
    forward(N, x, 1);
    const size_t cnt = (size_t)N->n * N->n * N->n * N->cout;
    if (cudaMemcpyAsync(y, N->yout, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, st) != cudaSuccess) throw 1;
  });
  N->st = keep;
  return r;
}

int unet_grid(const wbfbt_net* N) { return N->n; }
int unet_channels_in(const wbfbt_net* N) { return N->cin; }
int unet_channels_out(const wbfbt_net* N) { return N->cout; }
