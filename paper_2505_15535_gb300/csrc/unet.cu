// Learned preconditioner: a 3-level convolutional U-Net on the nodal grid, with BF16 weights
// and activations, FP32 accumulation and FP32 master weights trained by Adam.
//
// Network (channels C = 16, ReLU r; grids M0 = M, M1 = (M0-1)/2+1, M2 = (M1-1)/2+1):
//   a0 = r(conv(x)) 3->C;  s0 = r(conv(a0));  d1 = r(down(s0));  s1 = r(conv(d1));
//   d2 = r(down(s1));  m2 = r(conv(d2));  u1 = r(up(m2) + s1);  t1 = r(conv(u1));
//   u0 = r(up(t1) + s0);  t0 = r(conv(u0));  y = conv(t0) C->3
// with 3x3x3 zero-padded cross-correlations: conv (stride 1), down (stride 2) and up (the
// transposed stride-2 convolution).  Activations are channels-last [voxel][16] BF16 (32 B
// per voxel, one DRAM sector); inputs and outputs with 3 channels are padded to 16 with
// zero weights.  Every convolution is an implicit GEMM on the tensor cores, BF16 -> FP32:
//   stride-1 forward/backward-data (k_conv_tc), the stride-2 down-convolution and the up
//   layers' backward-data (k_down_tc), and the transposed stride-2 convolution (k_up_tc):
//   tcgen05 MMAs with accumulators in tensor memory, M = 128 positions, K = 16 input
//   channels, N = output channels (stacked over dz in the streaming forms);
//   weight gradients (k_wgrad_s1, k_wgrad_s2): mma.sync m16n8k16, partial sums per block,
//   reduced in a fixed order.
#include <cuda.h>  // CUtensorMap and the encoder's types; the encoder itself comes from the driver at run time
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "blas.h"
#include "internal.h"
#include "unet.h"

namespace nhmf {
namespace {

constexpr int kC = 16;
enum Gather { S1 = 0, DOWN2 = 1, UP2 = 2 };
enum Kind { CONV = 0, DOWN = 1, UP = 2 };
constexpr int kConvBlocks = 1216;  // elementwise kernels: 8 blocks of 256 per SM
constexpr int kWgBlocks = 608;     // weight-gradient partial blocks (4 per SM)
constexpr int kBgBlocks = 1216;    // bias-gradient partial blocks (8 per SM)

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

struct ConvArgs {
  const __nv_bfloat16* in;
  int m_in;
  const __nv_bfloat16* w;      // [27][16 co][16 ci]
  const float* bias;           // [16] or null (zero beyond cout)
  const __nv_bfloat16* add;    // [m_out^3][16] or null, added before the ReLU
  const __nv_bfloat16* mask;   // [m_out^3][16] or null, output zeroed where mask <= 0
  int relu;
  __nv_bfloat16* out;          // [m_out^3][16]
  float* out_planar;           // or [3][m_out^3] FP32 (channels 0..2)
  int m_out;
};

// Sum of the per-block weight-gradient partials [nblocks][27 * 256] in a fixed order (a block
// takes 32 consecutive entries, its 32 warps sum every 32nd partial block - coalesced rows -
// and one warp adds the 32 sums), written in the flat layout: conv/down W[o][c][tap] (a = o,
// b = c); up U[c][o][tap] (a = c, b = o).  With grad_b, one more block sums the per-block bias
// partials [nblocks][16] the same way.
__global__ void __launch_bounds__(1024) k_wgrad_reduce(const float* partial, const float* bpartial, int nblocks,
                                                       float* grad_w, float* grad_b, int kind, int cin, int cout) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  __shared__ float sh[32][33];
  if (blockIdx.x == 27 * 256 / 32) {  // the bias block
    const int ch = threadIdx.x & 15, g = threadIdx.x >> 4;  // 64 groups of 16 channels
    float s = 0.f;
    for (int b = g; b < nblocks; b += 64) s += bpartial[b * 16 + ch];
    float* flat = &sh[0][0];
    flat[g * 16 + ch] = s;
    __syncthreads();
    if (threadIdx.x < 16 && threadIdx.x < cout) {
      float t = 0.f;
      for (int j = 0; j < 64; ++j) t += flat[j * 16 + threadIdx.x];
      grad_b[threadIdx.x] = t;
    }
    return;
  }
  const int idx = blockIdx.x * 32 + tx;
  float s = 0.f;
  for (int b = ty; b < nblocks; b += 32) s += partial[(long long)b * 27 * 256 + idx];
  sh[ty][tx] = s;
  __syncthreads();
  if (ty != 0) return;
  s = 0.f;
#pragma unroll
  for (int j = 0; j < 32; ++j) s += sh[j][tx];
  const int tap = idx / 256, aa = (idx / 16) % 16, bb = idx % 16;
  if (kind == UP) {
    if (aa < cin && bb < cout) grad_w[((long long)aa * cout + bb) * 27 + tap] = s;
  } else {
    if (aa < cout && bb < cin) grad_w[((long long)aa * cin + bb) * 27 + tap] = s;
  }
}

// Bias gradient: per-block channel sums of P, then a fixed-order reduction.
// Per-block channel sums of P [voxel][16] (the bias gradient's partials): a thread adds whole
// 32-byte voxel rows, then the block adds its threads' sums in a fixed order.
__global__ void __launch_bounds__(256) k_bgrad_partial(const __nv_bfloat16* P, long long nvox, float* partial) {
  float s[16];
#pragma unroll
  for (int ch = 0; ch < 16; ++ch) s[ch] = 0.f;
  for (long long v = (long long)blockIdx.x * 256 + threadIdx.x; v < nvox; v += (long long)gridDim.x * 256) {
    const uint4* src = reinterpret_cast<const uint4*>(P + v * kC);
    const uint4 q0 = src[0], q1 = src[1];
    const uint32_t q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const __nv_bfloat162 x2 = *reinterpret_cast<const __nv_bfloat162*>(&q[h]);
      s[2 * h] += __low2float(x2);
      s[2 * h + 1] += __high2float(x2);
    }
  }
  __shared__ float sh[16][257];
#pragma unroll
  for (int ch = 0; ch < 16; ++ch) sh[ch][threadIdx.x] = s[ch];
  __syncthreads();
  __shared__ float sh2[16][17];
  {
    const int ch = threadIdx.x & 15, g = threadIdx.x >> 4;  // 16 groups of 16 threads
    float r = 0.f;
#pragma unroll
    for (int l = 0; l < 16; ++l) r += sh[ch][g * 16 + l];
    sh2[g][ch] = r;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    float r = 0.f;
#pragma unroll
    for (int g = 0; g < 16; ++g) r += sh2[g][threadIdx.x];
    partial[blockIdx.x * 16 + threadIdx.x] = r;
  }
}

// grad_b[ch] = sum over the partial blocks, in a fixed order (one block of 256 threads).
__global__ void __launch_bounds__(256) k_bgrad_reduce(const float* partial, int nblocks, float* grad_b, int cout) {
  const int ch = threadIdx.x & 15, g = threadIdx.x >> 4;
  float r = 0.f;
  for (int b = g; b < nblocks; b += 16) r += partial[b * 16 + ch];
  __shared__ float sh[16][17];
  sh[g][ch] = r;
  __syncthreads();
  if (threadIdx.x < 16 && threadIdx.x < cout) {
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) t += sh[j][threadIdx.x];
    grad_b[threadIdx.x] = t;
  }
}

// Forward and backward-data BF16 weights of one layer from the FP32 master weights.
__global__ void k_layer_weights(const float* w, int kind, int cin, int cout, __nv_bfloat16* wf, __nv_bfloat16* wb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 27 * 256) return;
  const int tap = idx / 256, co = (idx / 16) % 16, ci = idx % 16;
  float f = 0.f, b = 0.f;
  if (kind == UP) {
    // forward: co = o, ci = c: U[c][o][tap];  backward-data (DOWN2 gather): co = c, ci = o
    if (ci < cin && co < cout) f = w[((long long)ci * cout + co) * 27 + tap];
    if (co < cin && ci < cout) b = w[((long long)co * cout + ci) * 27 + tap];
  } else {
    // forward: W[o = co][c = ci][tap]; backward-data: co = c, ci = o, taps flipped for conv
    if (co < cout && ci < cin) f = w[((long long)co * cin + ci) * 27 + tap];
    const int tb = kind == CONV ? 26 - tap : tap;
    if (ci < cout && co < cin) b = w[((long long)ci * cin + co) * 27 + tb];
  }
  wf[idx] = __float2bfloat16(f);
  wb[idx] = __float2bfloat16(b);
}

__global__ void k_adam(long long n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

__device__ __forceinline__ bool constrained_dof(int bc, int c, long long v, int M) {
  const int vv = (int)v;  // grids of at most 785^3 nodes
  const int i = vv % M, k = vv / (M * M);
  if (bc == NHMF_BC_CLAMP_X0) return i == 0;
  if (bc == NHMF_BC_COMPRESSION) return k == 0 || (c == 2 && k == M - 1);
  return false;
}

// Network input: x16[v][c] = scale * src[c][v] (c < 3), 0 for c >= 3; scale = mul / (*den)
// when den is given, else mul.
template <typename TS>
__global__ void k_input(const TS* src, long long n, const double* den, double mul, __nv_bfloat16* x16) {
  const float s = float(den ? mul / *den : mul);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    uint32_t w[8];
    w[0] = pack_bf16(__float2bfloat16(float(src[v]) * s), __float2bfloat16(float(src[n + v]) * s));
    w[1] = pack_bf16(__float2bfloat16(float(src[2 * n + v]) * s), __float2bfloat16(0.f));
    for (int q = 2; q < 8; ++q) w[q] = 0u;
    uint4* dst = reinterpret_cast<uint4*>(x16 + v * kC);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

// Masked loss sums: partials of ||f (y - e)||^2 and ||f e||^2.
__global__ void __launch_bounds__(kRedThreads) k_loss_partials(const float* y, const float* e, long long n, int bc,
                                                               int M, double* partials) {
  // per thread in FP32 (a few dozen terms: relative error ~1e-6, exact for integer data), then
  // FP64 across threads and blocks
  float numf = 0.f, denf = 0.f;
  const int nn = (int)n, MM = M * M;  // grids of at most 785^3 nodes
  for (int v = blockIdx.x * kRedThreads + threadIdx.x; v < nn; v += kRedBlocks * kRedThreads) {
    const int i = v % M, k = v / MM;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const bool fixed = bc == NHMF_BC_CLAMP_X0 ? i == 0 : bc == NHMF_BC_COMPRESSION && (k == 0 || (c == 2 && k == M - 1));
      if (fixed) continue;
      const float ev = e[(long long)c * n + v], d = y[(long long)c * n + v] - ev;
      numf = fmaf(d, d, numf);
      denf = fmaf(ev, ev, denf);
    }
  }
  double num = numf, den = denf;
  __shared__ double sh[2][kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = num;
    sh[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) {
      a += sh[0][w];
      b += sh[1][w];
    }
    partials[blockIdx.x] = a;
    partials[kRedBlocks + blockIdx.x] = b;
  }
}

// Sums of the kRedBlocks loss partials in a fixed order (one block of kRedThreads threads).
__global__ void __launch_bounds__(kRedThreads) k_loss_final(const double* partials, double* num, double* den,
                                                            double* loss_acc) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) {
    a += partials[i];
    b += partials[kRedBlocks + i];
  }
  __shared__ double sh[2][kRedThreads];
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int st = kRedThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *num = sh[0][0];
    *den = sh[1][0];
    if (loss_acc) *loss_acc += sh[1][0] > 0.0 ? sh[0][0] / sh[1][0] : 0.0;
  }
}

// dy16[v][c] = 2 f (y - e) / den for c < 3, 0 otherwise.
__global__ void k_loss_grad(const float* y, const float* e, long long n, int bc, int M, const double* den,
                            __nv_bfloat16* dy16) {
  const float s = float(2.0 / *den);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    float d[3];
    for (int c = 0; c < 3; ++c)
      d[c] = constrained_dof(bc, c, v, M) ? 0.f : s * (y[c * n + v] - e[c * n + v]);
    uint4* dst = reinterpret_cast<uint4*>(dy16 + v * kC);
    dst[0] = make_uint4(pack_bf16(__float2bfloat16(d[0]), __float2bfloat16(d[1])),
                        pack_bf16(__float2bfloat16(d[2]), __float2bfloat16(0.f)), 0u, 0u);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// z = mask(y) * mul * (*scale) as FP64 (the preconditioner output); z_D = 0.
__global__ void k_output(const float* y, long long n, int bc, int M, const double* scale, double mul, double* z) {
  const double s = scale ? mul * *scale : mul;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * n; i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i / n);
    z[i] = constrained_dof(bc, c, i % n, M) ? 0.0 : s * double(y[i]);
  }
}

// pair slot <- (src * mul / *den) as FP32
__global__ void k_store_scaled(const double* src, long long n3, const double* den, double mul, float* dst) {
  const double s = mul / *den;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    dst[i] = float(src[i] * s);
}

const int kLayerKind[11] = {CONV, CONV, DOWN, CONV, DOWN, CONV, UP, CONV, UP, CONV, CONV};
const int kLayerCin[11] = {3, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16};
const int kLayerCout[11] = {16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 3};
enum { L_IN = 0, L_E0, L_D1, L_E1, L_D2, L_M2, L_U1, L_T1, L_U0, L_T0, L_OUT };

// ------------------------------------------------------------------ stride-1 conv on tcgen05
// Implicit GEMM on the fifth-generation tensor cores with the accumulator in tensor memory.
// A tile is 128 consecutive positions p of one z-plane in x-padded row order (row length
// R = m + 2, p = y R + x + 1; positions on the two pad columns are computed and dropped), so
// that tap (dx, dy, dz) reads a contiguous 128-row window of the staged plane z + dz: rows
// (p - p0) + R + 1 + dx + dy R of the padded positions p0 - 1 .. p0 + 128 + 2R (L = 130 + 2R
// rows, zero outside the grid).  A staged plane is kept as two arrays of 16-byte halves
// (channels 0-7, then 8-15, L rows apart), so that 8 consecutive rows form one canonical
// K-major core matrix (8 rows x 16 B, no swizzle).  A block walks a column of up to kTcZ tiles
// along z (fewer on small grids); MMAs are M = 128 positions x N output columns x K = 16 input
// channels, BF16 -> FP32 in tensor memory, issued by one thread, and each warp reads its 32
// accumulator rows back.
constexpr int kTcThreads = 128;
constexpr int kTcZ = 8;                       // at most this many tiles per block column along z
constexpr int kTcUnits = 600;                 // shorter columns below this many column units
constexpr unsigned kTcSpinLimit = 1u << 22;   // bounded wait for the MMAs of one tile
// instruction descriptor of kind::f16: D FP32 (bit 4), A and B BF16 (bits 7, 10), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, leading byte offset (between core
// matrices along K), stride byte offset (between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of an M = 128 MMA with N output columns (a multiple of 16, <= 256)
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

// D[tmem] (+)= A B for one 128 x N x 16 tile (N = 16 unless idesc says otherwise); issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, bool accumulate,
                                       uint32_t idesc = kTcIdesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)accumulate) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the phase `parity` of an mbarrier; returns whether it completed.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (unsigned it = 0; it < kTcSpinLimit && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// `cols` TMEM columns and `nbar` consecutive mbarriers (8 bytes apart) for the block.
__device__ __forceinline__ uint32_t tc_alloc_init(uint32_t* tslot, uint32_t bar, int nbar, uint32_t cols) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < nbar; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar + 8u * (uint32_t)i), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_sync();
  return *tslot;
}

// Block setup: weights [27][16 co][16 ci] to the canonical per-tap layout (co, ci) at
// (co % 8) 16 + (co / 8) 128 + (ci % 8) 2 + (ci / 8) 256, `cols` TMEM columns, the mbarrier.
__device__ __forceinline__ uint32_t tc_setup(const __nv_bfloat16* w, unsigned char* sB, uint32_t* tslot,
                                             uint32_t bar, uint32_t cols) {
  const uint4* wg = reinterpret_cast<const uint4*>(w);
  for (int i = threadIdx.x; i < 27 * 16 * 2; i += blockDim.x) {
    const int tap = i >> 5, co = (i >> 1) & 15, hf = i & 1;
    *reinterpret_cast<uint4*>(sB + tap * 512 + (co & 7) * 16 + (co >> 3) * 128 + hf * 256) = wg[i];
  }
  return tc_alloc_init(tslot, bar, 1, cols);
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t cols, bool timed_out, unsigned* status) {
  tc_sync();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
  if (timed_out && threadIdx.x == 0) atomicOr(status, kStatusTcTimeout);
}

// Skip-connection and mask rows of voxel v (32 bytes each), or zeros where absent.
__device__ __forceinline__ void tc_load_addmask(const ConvArgs& a, long long v, uint4 (&ad)[2], uint4 (&mk)[2]) {
  ad[0] = ad[1] = mk[0] = mk[1] = make_uint4(0u, 0u, 0u, 0u);
  if (a.add) {
    const uint4* ap = reinterpret_cast<const uint4*>(a.add + v * kC);
    ad[0] = ap[0];
    ad[1] = ap[1];
  }
  if (a.mask) {
    const uint4* mp = reinterpret_cast<const uint4*>(a.mask + v * kC);
    mk[0] = mp[0];
    mk[1] = mp[1];
  }
}

// Epilogue of one output voxel v from its 16 FP32 accumulators: + bias + add, ReLU, mask, store.
__device__ __forceinline__ void tc_emit(const ConvArgs& a, long long v, long long nvox, const uint32_t (&r)[16],
                                        const float* bias, const uint4 (&ad)[2], const uint4 (&mk)[2]) {
  float o[16];
#pragma unroll
  for (int ch = 0; ch < 16; ++ch) o[ch] = __uint_as_float(r[ch]) + (bias ? bias[ch] : 0.f);
  if (a.add) {
    const uint32_t q[8] = {ad[0].x, ad[0].y, ad[0].z, ad[0].w, ad[1].x, ad[1].y, ad[1].z, ad[1].w};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const __nv_bfloat162 x2 = *reinterpret_cast<const __nv_bfloat162*>(&q[h]);
      o[2 * h] += __low2float(x2);
      o[2 * h + 1] += __high2float(x2);
    }
  }
  if (a.relu) {
#pragma unroll
    for (int ch = 0; ch < 16; ++ch) o[ch] = fmaxf(o[ch], 0.f);
  }
  if (a.mask) {
    const uint32_t q[8] = {mk[0].x, mk[0].y, mk[0].z, mk[0].w, mk[1].x, mk[1].y, mk[1].z, mk[1].w};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const __nv_bfloat162 x2 = *reinterpret_cast<const __nv_bfloat162*>(&q[h]);
      if (!(__low2float(x2) > 0.f)) o[2 * h] = 0.f;
      if (!(__high2float(x2) > 0.f)) o[2 * h + 1] = 0.f;
    }
  }
  if (a.out_planar) {
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) a.out_planar[ch * nvox + v] = o[ch];
  } else {
    uint32_t pk[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(o[2 * h], o[2 * h + 1]);
      pk[h] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    uint4* dst = reinterpret_cast<uint4*>(a.out + v * kC);
    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  }
}

// 16-byte global -> shared copy on the cp.async path; `bytes` = 0 zero-fills the destination.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(__cvta_generic_to_global(src)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage positions base .. base + L - 1 of plane zz in a padded row order of length R with the
// grid at x in [xo, xo + m), y in [yo, yo + m) (zeros elsewhere) into `slot` (two 16-byte
// channel halves, L rows apart) with cp.async, as one commit group; the caller waits for the
// group (cp.async.wait_group / wait_all) and, before MMAs read the slot, fences the async proxy.
// Threads tid = 0 .. nthr - 1 of the block take rows tid, tid + nthr, ...
__device__ __forceinline__ void tc_stage_async(const __nv_bfloat16* __restrict__ in, int m, int R, int L, int base,
                                               int xo, int yo, int zz, unsigned char* slot, int tid, int nthr) {
  const uint32_t s = smem_u32(slot);
  const uint4* g = reinterpret_cast<const uint4*>(in);
  const bool plane_in = zz >= 0 && zz < m;
  // padded row and column of position base + j (base >= -R), stepped without division
  int yr = (base + tid + R) / R - 1, xr = (base + tid + R) % R;
  for (int j = tid; j < L; j += nthr) {
    const int y = yr - yo, x = xr - xo;
    const uint4* src = g;  // a valid address for the zero-filled copies, which read nothing
    uint32_t bytes = 0;
    if (plane_in && y >= 0 && y < m && x >= 0 && x < m) {
      src = g + 2 * (x + (long long)m * (y + (long long)m * zz));
      bytes = 16;
    }
    cp_async16(s + (uint32_t)j * 16u, src, bytes);
    cp_async16(s + (uint32_t)(L + j) * 16u, src + 1, bytes);
    xr += nthr;
    while (xr >= R) {
      xr -= R;
      ++yr;
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Plane-streaming form.  A block keeps the accumulators of all (up to kTcZ) output tiles of its
// column in tensor memory (16 columns each) and passes each input plane zi of the column's
// window (zb - 1 .. ze, inside the grid) through the tensor cores once: for each in-plane tap
// (dx, dy) one MMA of N = 16, 32 or 48 multiplies the plane's shifted 128-row window by the
// weights of dz = +1, 0, -1 stacked along N, and so adds plane zi's contribution to outputs
// zi - 1, zi, zi + 1 at once (those inside the column).  Each A tile is read 9 times per plane
// instead of 27 times per output tile.  The weights of each (dx, dy) form a 48-row strip, row
// 16 b + co holding dz = 1 - b, so that the rows of any run of consecutive outputs are one
// window of the strip.  Every output receives its 27 taps in the order of the per-tap form
// (dz, then dy, then dx) on a zeroed accumulator.
//
// Planes arrive by TMA (cp.async.bulk.tensor, 5-D map [z][y][x][2 halves][8 channels]): per
// 16-byte channel half one box of NY whole padded rows, x from x0 - 1 to x0 + W and zero
// outside the grid, so that staged row r of a half is padded position Yb R + r (Yb = the padded
// row of the tile's first halo position p0 - 1).  The grid runs as x-strips of W <=
// kConvStripMax columns (R = W + 2; a strip's halo columns hold the neighbouring strip's data),
// which keeps the boxes within the 256-element limit and the slots small (four blocks per SM).
// One thread of warp 4 waits for plane zi's box, issues its 9 MMAs and, once plane zi - 1's
// MMAs are done, refills that slot with plane zi + 2 (three slots); warps 0-3 zero a column's
// accumulators and read output zi - 2 back while plane zi's MMAs run.
constexpr int kTcSCols = 16 * kTcZ;               // TMEM columns: one 16-column accumulator per output tile
constexpr size_t kTcSSmemMin = 48 * 1024;         // at most 4 blocks (4 x 128 TMEM columns) per SM
constexpr int kTcSlots = 3;
#ifndef NHMF_CONV_STRIP
#define NHMF_CONV_STRIP 64
#endif
constexpr int kConvStripMax = NHMF_CONV_STRIP;    // widest x-strip
constexpr int kTcSThreads = 160;                  // warps 0-3: accumulators; warp 4: TMA and MMA issue

__device__ __forceinline__ void tc_st16_zero(uint32_t taddr) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(0u) : "memory");
}

// Weights [27][16 co][16 ci] as 9 strips of 48 rows: strip s = tap % 9 (dx, dy), row r =
// 16 (2 - tap / 9) + co, canonical K-major at (r % 8) 16 + (r / 8) 128 + (ci / 8) 768.
__device__ __forceinline__ void tc_weights_strips(const __nv_bfloat16* w, unsigned char* sB) {
  const uint4* wg = reinterpret_cast<const uint4*>(w);
  for (int i = threadIdx.x; i < 27 * 16 * 2; i += blockDim.x) {
    const int tap = i >> 5, co = (i >> 1) & 15, hf = i & 1, r = 16 * (2 - tap / 9) + co;
    *reinterpret_cast<uint4*>(sB + (tap % 9) * 1536 + (r & 7) * 16 + (r >> 3) * 128 + hf * 768) = wg[i];
  }
}

// x-strips of a stride-1 conv on an m^3 grid: count and width.
int conv_strip_width(int m, int* nstrips) {
  *nstrips = (m + kConvStripMax - 1) / kConvStripMax;
  return (m + *nstrips - 1) / *nstrips;
}

// Padded rows per box: a tile's taps read rows up to 128 + 3 R - 1 past the box start.
__host__ __device__ inline int tma_ny(int R) { return (128 + 3 * R) / R + 1; }
// Bytes of one staged channel half (NY R rows of 16 bytes), rounded up to 128.
__host__ __device__ inline uint32_t tma_h(int R) { return (uint32_t)((tma_ny(R) * R * 16 + 127) / 128 * 128); }

size_t conv_tc_smem(int m) {
  int ns = 0;
  const int W = conv_strip_width(m, &ns);
  const size_t need = 9 * 1536 + kTcSlots * 2 * (size_t)tma_h(W + 2) + 8 * 5 + 8 + 64;
  return std::max(need, kTcSSmemMin);
}

// OR of `v` over warps 0-3 (named barrier 1, 128 threads).
__device__ __forceinline__ bool bar_or_128(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r) : "r"((uint32_t)v) : "memory");
  return r != 0;
}


__device__ __forceinline__ void tma_load5(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(kTcSThreads) k_conv_tc(const ConvArgs a, const __grid_constant__ CUtensorMap map,
                                                         int zc, int W, int nstrips, unsigned* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int m = a.m_out, R = W + 2, NY = tma_ny(R);
  const uint32_t H = tma_h(R);
  unsigned char* sB = sm;
  unsigned char* sA = sm + 9 * 1536;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sA + kTcSlots * 2 * H);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2 + kTcSlots);
  float* sbias = reinterpret_cast<float*>(bar + 3 + kTcSlots);
  const uint32_t s_done = smem_u32(bar), s_full = s_done + 16u;
  const int warp = threadIdx.x >> 5;
  const bool epi = warp < 4, issuer = threadIdx.x == 128;
  tc_weights_strips(a.w, sB);
  if (threadIdx.x < 16) sbias[threadIdx.x] = a.bias ? a.bias[threadIdx.x] : 0.f;
  const uint32_t tmem = tc_alloc_init(tslot, s_done, 2 + kTcSlots, kTcSCols);
  const uint32_t lanes = tmem + ((32u * (uint32_t)(warp & 3)) << 16);
  const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);
  const int per_plane = (m * R + 127) / 128, nzc = (m + zc - 1) / zc;
  const long long nunits = (long long)per_plane * nstrips * nzc, nvox = (long long)m * m * m;
  const uint32_t box_bytes = 2u * (uint32_t)(NY * R * 16);
  unsigned k = 0, kc = 0;
  uint32_t fpar = 0, fpend = 0;
  bool timed_out = false;
  auto plane_done = [&](unsigned kk) { return tc_wait(s_done + 8u * (kk & 1u), (kk >> 1) & 1u); };
  auto wait_plane = [&](unsigned kk) -> bool {
    bool done = true;
    if (threadIdx.x == 0) done = plane_done(kk);
    if (bar_or_128(!done)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return true;
  };
  auto sync_or = [&](bool fail) -> bool {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const bool any = __syncthreads_or(fail) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return any;
  };
  for (long long unit = blockIdx.x; unit < nunits && !timed_out; unit += gridDim.x) {
    const int p0 = int(unit % per_plane) * 128;
    const long long rest = unit / per_plane;
    const int x0 = int(rest % nstrips) * W, zb = int(rest / nstrips) * zc, ze = min(m, zb + zc);
    const int first = max(zb - 1, 0), last = min(ze, m - 1);
    const int Yb = (p0 - 1 + R) / R - 1;
    const int p = p0 + (int)threadIdx.x, y = p / R, xl = p % R - 1;
    const bool own = epi && p < m * R && xl >= 0 && xl < W && x0 + xl < m;
    const long long v0 = (x0 + xl) + (long long)m * y;
    auto stage = [&](int z) {
      const int sl = z % kTcSlots;
      const uint32_t fb = s_full + 8u * (uint32_t)sl, dst = sA0 + (uint32_t)sl * 2u * H;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(box_bytes) : "memory");
      tma_load5(dst, &map, 0, 0, x0 - 1, Yb - 1, z, fb);
      tma_load5(dst + H, &map, 0, 1, x0 - 1, Yb - 1, z, fb);
      fpend |= 1u << sl;
    };
    if (epi) {
      for (int c = 0; c < ze - zb; ++c) tc_st16_zero(lanes + 16u * (uint32_t)c);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    if (issuer) {
      stage(first);
      if (first + 1 <= last) stage(first + 1);
    }
    sync_or(false);
    for (int zi = first; zi <= last; ++zi, ++k) {
      bool fail = false;
      if (issuer) {
        const int sl = zi % kTcSlots;
        fail = !tc_wait(s_full + 8u * (uint32_t)sl, (fpar >> sl) & 1u);
        fpar ^= 1u << sl;
        fpend &= ~(1u << sl);
        if (!fail) {
          const int olo = max(zi - 1, zb), ohi = min(zi + 1, ze - 1), blo = 1 - zi + olo;
          const uint32_t idesc = tc_idesc(16 * (ohi - olo + 1)), acc = tmem + 16u * (uint32_t)(olo - zb);
          const uint64_t da = tc_desc(sA0 + (uint32_t)sl * 2u * H + (uint32_t)(p0 + R - Yb * R) * 16u, H, 128u);
          const uint64_t db = tc_desc(sB0 + 256u * (uint32_t)blo, 768u, 128u);
#pragma unroll
          for (int s = 0; s < 9; ++s) {
            const int dx = s % 3 - 1, dy = s / 3 - 1;
            tc_mma(acc, da + (uint64_t)(long long)(dx + dy * R), db + (uint64_t)(96 * s), true, idesc);
          }
          tc_commit(s_done + 8u * (k & 1u));
          kc = k + 1;
          if (zi + 2 <= last) {
            if (zi > first) fail = !plane_done(k - 1);
            if (!fail) stage(zi + 2);
          }
        }
      }
      if (epi && zi > first) {
        const int o = zi - 2;
        const bool emit = o >= zb && own;
        uint4 ad[2], mk[2];
        if (emit) tc_load_addmask(a, v0 + (long long)m * m * o, ad, mk);
        fail = !wait_plane(k - 1);
        if (!fail && o >= zb) {
          uint32_t r[16];
          tc_ld16(lanes + 16u * (uint32_t)(o - zb), r);
          if (emit) tc_emit(a, v0 + (long long)m * m * o, nvox, r, sbias, ad, mk);
        }
      }
      if (sync_or(fail)) { timed_out = true; break; }
    }
    if (!timed_out) {
      bool fail = false;
      if (epi) {
        fail = !wait_plane(k - 1);
        for (int o = max(zb, last - 1); o < ze && !fail; ++o) {
          uint32_t r[16];
          tc_ld16(lanes + 16u * (uint32_t)(o - zb), r);
          if (own) {
            uint4 ad[2], mk[2];
            tc_load_addmask(a, v0 + (long long)m * m * o, ad, mk);
            tc_emit(a, v0 + (long long)m * m * o, nvox, r, sbias, ad, mk);
          }
        }
      }
      if (sync_or(fail)) timed_out = true;
    }
  }
  if (issuer && timed_out) {
    for (int sl = 0; sl < kTcSlots; ++sl)
      if (fpend & (1u << sl)) tc_wait(s_full + 8u * (uint32_t)sl, (fpar >> sl) & 1u);
    if (kc > 0) plane_done(kc - 1);
  }
  tc_teardown(tmem, kTcSCols, timed_out, status);
}

// ------------------------------------------------------------------ stride-2 conv on tcgen05
// out[o] = sum_d W_d in[2 o + d] (the down-convolution and the up layers' backward-data) in the
// plane-streaming form of k_conv_tc, with planes staged by cp.async.  A tile is 128
// consecutive coarse positions of one output plane in x-padded row order (R = W + 2 for an
// x-strip of W coarse columns from x0).  A fine plane f is staged as four parity sub-planes
// (py, px): row j of a sub-plane is padded coarse position P0 + j = Y R + X (P0 = p0 - R - 1,
// L = R + 129 rows) and holds the fine voxel (2 (x0 + X - 1) + px, 2 Y + py, f), zero outside the
// grid, so that tap (dx, dy) reads a contiguous 128-row window of sub-plane (dy != 0, dx != 0)
// from row R + 1 + sx + sy R (s = -1 for d = -1, else 0).  Plane f adds to output f / 2 (dz = 0) if f is
// even and to outputs (f - 1) / 2 (dz = +1) and (f + 1) / 2 (dz = -1) if f is odd; the weights of
// each (dx, dy) are a strip of dz = +1, -1, 0 blocks, so one MMA of N = 16 or 32 per (dx, dy)
// covers the plane's outputs in the column.  Output o is complete after plane min(2 o + 1,
// m_in - 1) and is read back while later planes run.  One thread of warp 4 issues the MMAs;
// warps 0-3 stage planes two ahead (three slots) and read accumulators back.
constexpr int kDnStripMax = 32;
#ifndef NHMF_DN_SLOTS
#define NHMF_DN_SLOTS 3
#endif
constexpr int kDnSlots = NHMF_DN_SLOTS;  // planes staged up to kDnSlots - 1 ahead

// Wait until at most n (0 .. 3) of this thread's cp.async groups are pending.
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  if (n <= 0)
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  else if (n == 1)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
  else if (n == 2)
    asm volatile("cp.async.wait_group 2;" ::: "memory");
  else
    asm volatile("cp.async.wait_group 3;" ::: "memory");
}

__device__ __forceinline__ void dn_weights_strips(const __nv_bfloat16* w, unsigned char* sB) {
  const uint4* wg = reinterpret_cast<const uint4*>(w);
  for (int i = threadIdx.x; i < 27 * 16 * 2; i += blockDim.x) {
    const int tap = i >> 5, co = (i >> 1) & 15, hf = i & 1, dz = tap / 9 - 1;
    const int r = 16 * (dz == 1 ? 0 : (dz == -1 ? 1 : 2)) + co;
    *reinterpret_cast<uint4*>(sB + (tap % 9) * 1536 + (r & 7) * 16 + (r >> 3) * 128 + hf * 768) = wg[i];
  }
}

// Fine plane f into `slot` ([4 sub-planes][2 halves][L][16 B]) by threads tid = 0 .. nthr - 1.
__device__ __forceinline__ void dn_stage_async(const __nv_bfloat16* __restrict__ in, int mi, int R, int L, int P0,
                                               int x0, int f, unsigned char* slot, int tid, int nthr) {
  const uint32_t s = smem_u32(slot);
  const uint4* g = reinterpret_cast<const uint4*>(in);
  const bool plane_in = f >= 0 && f < mi;
  int Yr = (P0 + tid + 2 * R) / R - 2, Xr = (P0 + tid + 2 * R) % R;  // row and column of P0 + j (P0 >= -R - 1)
  for (int j = tid; j < L; j += nthr) {
    const int cx = 2 * (Xr - 1 + x0), cy = 2 * Yr;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      const int fx = cx + (sp & 1), fy = cy + (sp >> 1);
      const uint4* src = g;  // a valid address for the zero-filled copies
      uint32_t bytes = 0;
      if (plane_in && fx >= 0 && fx < mi && fy >= 0 && fy < mi) {
        src = g + 2 * (fx + (long long)mi * (fy + (long long)mi * f));
        bytes = 16;
      }
      cp_async16(s + (uint32_t)((2 * sp) * L + j) * 16u, src, bytes);
      cp_async16(s + (uint32_t)((2 * sp + 1) * L + j) * 16u, src + 1, bytes);
    }
    Xr += nthr;
    while (Xr >= R) {
      Xr -= R;
      ++Yr;
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

size_t down_tc_smem(int W) {
  const int L = W + 2 + 129;
  const size_t need = 9 * 1536 + (size_t)kDnSlots * 4 * 2 * L * 16 + 8 * 2 + 8 + 64;
  return std::max(need, kTcSSmemMin);
}

__global__ void __launch_bounds__(kTcSThreads) k_down_tc(const ConvArgs a, int zc, int W, int nstrips,
                                                         unsigned* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int mo = a.m_out, mi = a.m_in, R = W + 2, L = R + 129;
  const uint32_t slot_bytes = 4u * 2u * (uint32_t)L * 16u;
  unsigned char* sB = sm;                                  // [9 strips][1536 B] weights
  unsigned char* sA = sm + 9 * 1536;                       // [kDnSlots][4 sub-planes][2 halves][L][16 B]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sA + kDnSlots * slot_bytes);  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  float* sbias = reinterpret_cast<float*>(bar + 3);        // [16]
  const uint32_t s_done = smem_u32(bar);
  const int warp = threadIdx.x >> 5;
  const bool epi = warp < 4, issuer = threadIdx.x == 128;
  auto slot = [&](int f) { return sA + (f % kDnSlots) * slot_bytes; };  // f >= 0
  dn_weights_strips(a.w, sB);
  if (threadIdx.x < 16) sbias[threadIdx.x] = a.bias ? a.bias[threadIdx.x] : 0.f;
  const uint32_t tmem = tc_alloc_init(tslot, s_done, 2, kTcSCols);  // synchronises the block
  const uint32_t lanes = tmem + ((32u * (uint32_t)(warp & 3)) << 16);
  const uint32_t sB0 = smem_u32(sB);

  const int per_plane = (mo * R + 127) / 128, nzc = (mo + zc - 1) / zc;
  const long long nunits = (long long)per_plane * nstrips * nzc, nvox = (long long)mo * mo * mo;
  unsigned k = 0, kc = 0;  // planes issued: plane kk commits to mbarrier kk & 1, phase kk >> 1
  bool timed_out = false;
  auto plane_done = [&](unsigned kk) { return tc_wait(s_done + 8u * (kk & 1u), (kk >> 1) & 1u); };
  auto wait_plane = [&](unsigned kk) -> bool {
    bool done = true;
    if (threadIdx.x == 0) done = plane_done(kk);
    if (bar_or_128(!done)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return true;
  };
  auto sync_or = [&](bool fail) -> bool {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const bool any = __syncthreads_or(fail) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return any;
  };
  for (long long unit = blockIdx.x; unit < nunits && !timed_out; unit += gridDim.x) {
    const int p0 = int(unit % per_plane) * 128;
    const long long rest = unit / per_plane;
    const int x0 = int(rest % nstrips) * W, zb = int(rest / nstrips) * zc, ze = min(mo, zb + zc);
    const int ffirst = max(2 * zb - 1, 0), flast = min(2 * ze - 1, mi - 1);  // fine planes of the column
    const int p = p0 + (int)threadIdx.x, y = p / R, xl = p % R - 1;
    const bool own = epi && p < mo * R && xl >= 0 && xl < W && x0 + xl < mo;
    const long long v0 = (x0 + xl) + (long long)mo * y;
    auto finish = [&](int o) {
      uint32_t r[16];
      tc_ld16(lanes + 16u * (uint32_t)(o - zb), r);
      if (own) {
        uint4 ad[2], mk[2];
        tc_load_addmask(a, v0 + (long long)mo * mo * o, ad, mk);
        tc_emit(a, v0 + (long long)mo * mo * o, nvox, r, sbias, ad, mk);
      }
    };
    if (epi) {
      for (int c = 0; c < ze - zb; ++c) tc_st16_zero(lanes + 16u * (uint32_t)c);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      const int fpre = min(ffirst + kDnSlots - 2, flast);
      for (int f = ffirst; f <= fpre; ++f)
        dn_stage_async(a.in, mi, R, L, p0 - R - 1, x0, f, slot(f), threadIdx.x, 128);
      cp_async_wait_pending(fpre - ffirst);  // plane ffirst has landed
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    sync_or(false);
    int next_out = zb;  // the next output plane to read back
    for (int f = ffirst; f <= flast; ++f, ++k) {
      if (issuer) {
        int olo, nb, blo;
        if ((f & 1) == 0) {
          olo = f / 2, nb = 1, blo = 2;
        } else {
          const bool lo_in = (f - 1) / 2 >= zb, hi_in = (f + 1) / 2 < ze;
          olo = lo_in ? (f - 1) / 2 : (f + 1) / 2;
          nb = (lo_in && hi_in) ? 2 : 1;
          blo = lo_in ? 0 : 1;
        }
        const uint32_t idesc = tc_idesc(16 * nb), acc = tmem + 16u * (uint32_t)(olo - zb);
        const uint32_t sa = smem_u32(slot(f)), sb = sB0 + 256u * (uint32_t)blo;
#pragma unroll
        for (int s9 = 0; s9 < 9; ++s9) {
          const int dx = s9 % 3 - 1, dy = s9 / 3 - 1;
          const int sp = (dy != 0 ? 2 : 0) + (dx != 0 ? 1 : 0);
          const int j0 = R + 1 + (dx < 0 ? -1 : 0) + (dy < 0 ? -R : 0);
          tc_mma(acc, tc_desc(sa + (uint32_t)(2 * sp * L + j0) * 16u, (uint32_t)(L * 16), 128u),
                 tc_desc(sb + 1536u * (uint32_t)s9, 768u, 128u), true, idesc);
        }
        tc_commit(s_done + 8u * (k & 1u));
        kc = k + 1;
      }
      bool fail = false;
      if (epi) {
        fail = f > ffirst && !wait_plane(k - 1);
        if (!fail) {
          // plane f - 1's MMAs are done: its slot takes plane f + kDnSlots - 1, and the outputs
          // whose last plane is at most f - 1 are complete
          const int fa = f + kDnSlots - 1;
          if (fa <= flast) dn_stage_async(a.in, mi, R, L, p0 - R - 1, x0, fa, slot(fa), threadIdx.x, 128);
          while (f > ffirst && next_out < ze && min(2 * next_out + 1, mi - 1) <= f - 1) finish(next_out++);
          cp_async_wait_pending(min(fa, flast) - f - 1);  // plane f + 1 has landed
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
      }
      if (sync_or(fail)) {
        timed_out = true;
        break;
      }
    }
    if (!timed_out) {
      bool fail = false;
      if (epi) {
        fail = !wait_plane(k - 1);
        while (!fail && next_out < ze) finish(next_out++);
      }
      if (sync_or(fail)) timed_out = true;
    }
  }
  if (epi) cp_async_wait_all();
  if (issuer && timed_out && kc > 0) plane_done(kc - 1);  // MMAs still in flight end before TMEM is freed
  tc_teardown(tmem, kTcSCols, timed_out, status);
}

// ------------------------------------------------------------------ transposed stride-2 conv on tcgen05
// out[o] = sum over taps d with o - d even of W_d in[(o - d) / 2], per direction.  Writing
// o = 2c + q (q = 0, 1), class q = 0 takes tap d = 0 (source c) and q = 1 takes d = -1 (source
// c + 1) and d = +1 (source c): the 8 parity classes are convolutions on the coarse grid with
// 1, 2, 4 or 8 taps of source shifts in {0, 1}^3, 27 taps in all.  A tile is 128 consecutive
// coarse positions p = y R + x (R = m_in + 1, x = m_in is a zero pad column) of coarse plane
// c_z; shift (sx, sy) reads rows (p - p0) + sx + sy R of the staged plane c_z + sz (L = 129 + R
// rows).  The 8 classes accumulate in 8 groups of 16 TMEM columns; one commit covers the 27
// MMAs and the epilogue writes the 8 fine voxels of each coarse position.  Planes c_z, c_z + 1
// are staged in a ring of three slots, c_z + 2 while the MMAs of c_z run.
constexpr int kUpCols = 128;
constexpr size_t kUpSmemMin = 52 * 1024;  // at most 4 blocks (4 x 128 TMEM columns) per SM

size_t up_tc_smem(int mi) {
  const size_t need = 27 * 512 + 3 * 2 * (size_t)(129 + mi + 1) * 16 + 16 + 64;
  return std::max(need, kUpSmemMin);
}

__global__ void __launch_bounds__(kTcThreads, 4) k_up_tc(const ConvArgs a, int zc, unsigned* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int mi = a.m_in, mo = a.m_out, R = mi + 1, L = 129 + R;
  unsigned char* sB = sm;
  unsigned char* sA = sm + 27 * 512;                       // [3 slots][2 halves][L][16 B]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sA + 6 * L * 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  float* sbias = reinterpret_cast<float*>(bar + 2);        // [16]
  const uint32_t s_bar = smem_u32(bar);
  const int warp = threadIdx.x >> 5;
  auto slot = [&](int plane) { return sA + (plane % 3) * 2 * L * 16; };  // plane >= 0
  if (threadIdx.x < 16) sbias[threadIdx.x] = a.bias ? a.bias[threadIdx.x] : 0.f;
  const uint32_t tmem = tc_setup(a.w, sB, tslot, s_bar, kUpCols);  // synchronises the block

  const int per_plane = (mi * R + 127) / 128, nzc = (mi + zc - 1) / zc;
  const long long nunits = (long long)per_plane * nzc, nvox = (long long)mo * mo * mo;
  uint32_t phase = 0;
  bool timed_out = false;
  for (long long unit = blockIdx.x; unit < nunits && !timed_out; unit += gridDim.x) {
    const int p0 = int(unit % per_plane) * 128, zb = int(unit / per_plane) * zc, ze = min(mi, zb + zc);
    // staged row j of a plane is coarse position p0 + j = y R + x
    for (int pl = zb; pl <= zb + 1; ++pl) tc_stage_async(a.in, mi, R, L, p0, 0, 0, pl, slot(pl), threadIdx.x, blockDim.x);
    cp_async_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    for (int cz = zb; cz < ze; ++cz) {
      if (threadIdx.x == 0) {
        const uint32_t b0 = smem_u32(sB);
        for (int cl = 0; cl < 8; ++cl) {
          const int qx = cl & 1, qy = (cl >> 1) & 1, qz = cl >> 2;
          int k = 0;
          for (int sz = 0; sz <= qz; ++sz)
            for (int sy = 0; sy <= qy; ++sy)
              for (int sx = 0; sx <= qx; ++sx, ++k) {
                // d = 0 for q = 0; for q = 1, shift 1 <-> d = -1 and shift 0 <-> d = +1
                const int dx = qx ? (sx ? -1 : 1) : 0, dy = qy ? (sy ? -1 : 1) : 0, dz = qz ? (sz ? -1 : 1) : 0;
                const int tap = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                const int j0 = sx + sy * R;  // rows j0 .. j0 + 127 < L of plane cz + sz
                tc_mma(tmem + (uint32_t)(16 * cl),
                       tc_desc(smem_u32(slot(cz + sz)) + (uint32_t)j0 * 16u, (uint32_t)(L * 16), 128u),
                       tc_desc(b0 + (uint32_t)tap * 512u, 256u, 128u), k > 0);
              }
        }
        tc_commit(s_bar);
      }
      // plane cz + 2 goes to the slot of plane cz - 1; the copy runs during the MMAs and the epilogue
      if (cz + 1 < ze) tc_stage_async(a.in, mi, R, L, p0, 0, 0, cz + 2, slot(cz + 2), threadIdx.x, blockDim.x);
      // row threadIdx.x is coarse position p; its fine voxels are the 8 classes (qx, qy, qz).  The
      // skip rows of classes 0-3 load while the MMAs run, those of 4-7 while 0-3 are written
      // (the mask, in the backward pass, is read at the store)
      const int p = p0 + threadIdx.x, y = p / R, x = p % R;
      const bool ok = p < mi * R && x < mi;
      auto fine = [&](int cl, long long& v) -> bool {
        const int qx = cl & 1, qy = (cl >> 1) & 1, qz = cl >> 2;
        v = (2 * x + qx) + (long long)mo * ((2 * y + qy) + (long long)mo * (2 * cz + qz));
        return ok && (!qx || x < mi - 1) && (!qy || y < mi - 1) && (!qz || cz < mi - 1);
      };
      auto load_skip = [&](int cl, uint4 (&q)[2]) {
        long long v;
        q[0] = q[1] = make_uint4(0u, 0u, 0u, 0u);
        if (a.add && fine(cl, v)) {
          const uint4* src = reinterpret_cast<const uint4*>(a.add + v * kC);
          q[0] = src[0];
          q[1] = src[1];
        }
      };
      auto store = [&](int cl, const uint4 (&q)[2]) {
        uint32_t r[16];
        tc_ld16(tmem + ((32u * (uint32_t)warp) << 16) + (uint32_t)(16 * cl), r);
        long long v;
        if (fine(cl, v)) {
          uint4 mk[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
          if (a.mask) {
            const uint4* src = reinterpret_cast<const uint4*>(a.mask + v * kC);
            mk[0] = src[0];
            mk[1] = src[1];
          }
          tc_emit(a, v, nvox, r, sbias, q, mk);
        }
      };
      uint4 pre[4][2];
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) load_skip(c4, pre[c4]);
      bool done = true;
      if (threadIdx.x == 0) done = tc_wait(s_bar, phase);
      phase ^= 1u;
      timed_out = __syncthreads_or(!done) != 0;
      if (timed_out) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        store(c4, pre[c4]);
        load_skip(c4 + 4, pre[c4]);
      }
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) store(c4 + 4, pre[c4]);
      cp_async_wait_all();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_sync();
    }
  }
  cp_async_wait_all();
  tc_teardown(tmem, kUpCols, timed_out, status);
}

// Weight gradient of the stride-1 gather, tiled: G[tap][a][b] = sum_v P[v][a] Q[v + d_tap][b].
// A block takes tiles of 128 consecutive positions of one z-plane of an x-strip in x-padded
// row order (as k_conv_tc) along a column in z.  It stages the tile's P rows and a ring of Q
// planes (the z - 1 .. z + 1 windows of all taps, zero outside the grid, the neighbouring
// strip's data in the halo columns) as 16-byte channel halves, so
// that every 8 x 8 block of a fragment is one ldmatrix: per chunk of 16 positions one
// ldmatrix.x4.trans gives the A fragment (P^T, channels a x positions) for all the warp's
// taps, and one per tap gives the B fragments (positions x channels b) of both n-tiles.
// 9 warps, warp w owns taps 3w..3w+2; per-block partials reduced by k_wgrad_reduce.
constexpr int kWgThreads = 288;

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

// Bias-gradient share of an A fragment (P^T, channels x 16 positions, m16n8k16 layout): lane
// (g, t) holds channels g (a0, a2) and g + 8 (a1, a3) at 4 of the positions.
__device__ __forceinline__ void frag_channel_sums(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, float& sg,
                                                  float& sg8) {
  const __nv_bfloat162 x0 = *reinterpret_cast<const __nv_bfloat162*>(&a0),
                       x1 = *reinterpret_cast<const __nv_bfloat162*>(&a1),
                       x2 = *reinterpret_cast<const __nv_bfloat162*>(&a2),
                       x3 = *reinterpret_cast<const __nv_bfloat162*>(&a3);
  sg += (__low2float(x0) + __high2float(x0)) + (__low2float(x2) + __high2float(x2));
  sg8 += (__low2float(x1) + __high2float(x1)) + (__low2float(x3) + __high2float(x3));
}
// All 9 warps: the block's 16 channel totals (per warp the 4 lanes of each channel, then the
// warps in order) to bpartial[blockIdx.x][16].  Ends with a block barrier.
__device__ __forceinline__ void bias_partial_store(float sg, float sg8, float* bpartial) {
  __shared__ float bsh[kWgThreads / 32][16];
  sg += __shfl_xor_sync(0xffffffffu, sg, 1);
  sg8 += __shfl_xor_sync(0xffffffffu, sg8, 1);
  sg += __shfl_xor_sync(0xffffffffu, sg, 2);
  sg8 += __shfl_xor_sync(0xffffffffu, sg8, 2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if ((lane & 3) == 0) {
    bsh[warp][lane >> 2] = sg;
    bsh[warp][(lane >> 2) + 8] = sg8;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kWgThreads / 32; ++w) t += bsh[w][threadIdx.x];
    bpartial[blockIdx.x * 16 + threadIdx.x] = t;
  }
}

size_t wgrad_s1_smem(int W) { return 2 * 2 * 128 * 16 + 4 * 2 * (size_t)(130 + 2 * (W + 2)) * 16; }

// P rows of a tile, asynchronously: position p0 + j = y R + xl + 1 of plane z in the x-strip
// of W columns from x0 (zero on the pad columns, past the strip or the grid) to row j of both
// 16-byte channel halves (128 rows apart).
__device__ __forceinline__ void wg_stage_rows_async(const __nv_bfloat16* __restrict__ P, int m, int R, int p0, int z,
                                                    int x0, int W, unsigned char* sP) {
  const uint32_t s = smem_u32(sP);
  const uint4* g = reinterpret_cast<const uint4*>(P);
  for (int j = threadIdx.x; j < 128; j += blockDim.x) {
    const int p = p0 + j, y = p / R, xl = p % R - 1, x = x0 + xl;
    const uint4* src = g;
    uint32_t bytes = 0;
    if (p < m * R && xl >= 0 && xl < W && x < m) {
      src = g + 2 * (x + (long long)m * (y + (long long)m * z));
      bytes = 16;
    }
    cp_async16(s + (uint32_t)j * 16u, src, bytes);
    cp_async16(s + (uint32_t)(128 + j) * 16u, src + 1, bytes);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

#ifndef NHMF_WG_MINB
#define NHMF_WG_MINB 4
#endif
__global__ void __launch_bounds__(kWgThreads, NHMF_WG_MINB) k_wgrad_s1(const __nv_bfloat16* __restrict__ P,
                                                         const __nv_bfloat16* __restrict__ Q, int m, int zc, int W,
                                                         int nstrips, float* partial, float* bpartial) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int R = W + 2, L = 130 + 2 * R;
  unsigned char* sP0 = sm;                      // [2 buffers][2 halves][128][16 B]
  unsigned char* sQ = sm + 2 * 2 * 128 * 16;    // [4 slots][2 halves][L][16 B]
  auto slot = [&](int plane) { return sQ + ((plane + 4) & 3) * 2 * L * 16; };  // plane >= -1
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int per_plane = (m * R + 127) / 128, nzc = (m + zc - 1) / zc;
  const long long nunits = (long long)per_plane * nstrips * nzc;
  float acc[3][2][4] = {};
  unsigned tt = 0;  // tiles done by this block; the P rows of tile tt are in buffer tt & 1
  float bsg = 0.f, bsg8 = 0.f;  // channels g, g + 8 of P over this warp's share of the chunks (bias gradient)
  unsigned chunk = 0;            // chunks of 16 positions done by this block; chunk % 9 adds its fragments
  // ldmatrix row of this lane: matrix lane / 8, row lane % 8
  const int lm = lane >> 3, lr = lane & 7;
  for (long long unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
    const int p0 = int(unit % per_plane) * 128;
    const long long rest = unit / per_plane;
    const int x0 = int(rest % nstrips) * W, zb = int(rest / nstrips) * zc, ze = min(m, zb + zc);
    // planes z - 1 .. z + 1 of Q and the P rows of plane z are in shared memory when tile z
    // starts; plane z + 2 and the rows of plane z + 1 are copied while tile z computes
    for (int pl = zb - 1; pl <= zb + 1; ++pl)
      tc_stage_async(Q, m, R, L, p0 - 1, 1 - x0, 1, pl, slot(pl), threadIdx.x, blockDim.x);
    wg_stage_rows_async(P, m, R, p0, zb, x0, W, sP0 + (tt & 1u) * 4096);
    cp_async_wait_all();
    __syncthreads();
    for (int z = zb; z < ze; ++z, ++tt) {
      if (z + 1 < ze) {
        tc_stage_async(Q, m, R, L, p0 - 1, 1 - x0, 1, z + 2, slot(z + 2), threadIdx.x, blockDim.x);
        wg_stage_rows_async(P, m, R, p0, z + 1, x0, W, sP0 + ((tt + 1) & 1u) * 4096);
      }
      const uint32_t sp = smem_u32(sP0 + (tt & 1u) * 4096);
      for (int c = 0; c < 8; ++c) {
        // A = P^T on positions 16c..16c+15: matrices (k 0-7, a lo), (k 0-7, a hi), (k 8-15, a lo), (k 8-15, a hi)
        uint32_t a0, a1, a2, a3;
        ldsm_x4_trans(sp + (uint32_t)(((lm & 1) * 128 + 16 * c + (lm >> 1) * 8 + lr) * 16), a0, a1, a2, a3);
#pragma unroll
        for (int jt = 0; jt < 3; ++jt) {
          const int tap = 3 * warp + jt;
          const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
          const int row = R + 1 + dx + dy * R + 16 * c;  // staged row of position 16c of plane z + dz
          // B: matrices (k 0-7, b lo), (k 8-15, b lo), (k 0-7, b hi), (k 8-15, b hi)
          uint32_t b0, b1, b2, b3;
          ldsm_x4_trans(smem_u32(slot(z + dz)) + (uint32_t)(((lm >> 1) * L + row + (lm & 1) * 8 + lr) * 16), b0, b1,
                        b2, b3);
          mma16816(acc[jt][0], a0, a1, a2, a3, b0, b1);
          mma16816(acc[jt][1], a0, a1, a2, a3, b2, b3);
        }
        // the bias gradient's share, after the MMAs have consumed the fragment
        if (bpartial && chunk % (kWgThreads / 32) == (unsigned)warp) frag_channel_sums(a0, a1, a2, a3, bsg, bsg8);
        ++chunk;
      }
      cp_async_wait_all();
      __syncthreads();
    }
  }
  if (bpartial) bias_partial_store(bsg, bsg8, bpartial);
  float* out = partial + (long long)blockIdx.x * 27 * 256;
#pragma unroll
  for (int jt = 0; jt < 3; ++jt) {
    const int tap = 3 * warp + jt;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int b = 8 * h + 2 * t;
      out[tap * 256 + g * 16 + b] = acc[jt][h][0];
      out[tap * 256 + g * 16 + b + 1] = acc[jt][h][1];
      out[tap * 256 + (g + 8) * 16 + b] = acc[jt][h][2];
      out[tap * 256 + (g + 8) * 16 + b + 1] = acc[jt][h][3];
    }
  }
}

// Weight gradient of the stride-2 gather (the down-convolution), tiled like k_wgrad_s1:
// G[tap][a][b] = sum_v P[v][a] Q[2 v + d_tap][b] over the coarse grid (Q on the fine grid,
// zero outside it).  A unit is a segment of `seg` coarse voxels (a multiple of 16, zero past
// the grid) of one coarse row cy, along a column of zc coarse planes.  Per coarse plane cz it
// stages the segment's P rows and, of fine planes 2 cz - 1 .. 2 cz + 1, the fine rows 2 cy - 1
// .. 2 cy + 1 over fine x 2 x0 - 1 .. 2 (x0 + seg) - 1 (Wf = 2 seg + 1 positions per row), as
// 16-byte channel halves, in a ring of five fine-plane slots: the two fine planes of the next
// coarse plane and its P rows are copied while this one computes.  The A fragment (P^T) comes
// from ldmatrix.trans as in k_wgrad_s1; the B rows of position k and tap (dx, dy) are the
// staged fine voxels 2 k + dx + 1 of row dy + 1, one ldmatrix row address per lane.
constexpr int kW2Seg = 80;     // widest segment
constexpr int kW2Slots = 5;

int wgrad_s2_seg(int mp, int* nseg) {
  *nseg = (mp + kW2Seg - 1) / kW2Seg;
  return ((mp + *nseg - 1) / *nseg + 15) / 16 * 16;
}
size_t wgrad_s2_smem(int seg) { return 2 * 2 * (size_t)seg * 16 + kW2Slots * 2 * 3 * (size_t)(2 * seg + 1) * 16; }

__global__ void __launch_bounds__(kWgThreads) k_wgrad_s2(const __nv_bfloat16* __restrict__ P, int mp,
                                                         const __nv_bfloat16* __restrict__ Q, int mq, int seg,
                                                         int nseg, int zc, float* partial, float* bpartial) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int Wf = 2 * seg + 1, hs = 3 * Wf * 16;  // bytes per staged fine half
  unsigned char* sP0 = sm;                        // [2 buffers][2 halves][seg][16 B]
  unsigned char* sQ = sm + 2 * 2 * seg * 16;      // [kW2Slots][2 halves][3 rows][Wf][16 B]
  auto slot = [&](int f) { return sQ + ((f + kW2Slots) % kW2Slots) * 2 * hs; };  // fine plane f >= -1
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int lm = lane >> 3, lr = lane & 7;
  const uint4* qg = reinterpret_cast<const uint4*>(Q);
  const uint4* pg = reinterpret_cast<const uint4*>(P);
  const int nzc = (mp + zc - 1) / zc;
  const long long nunits = (long long)mp * nseg * nzc;
  float acc[3][2][4] = {};
  unsigned tt = 0;  // coarse planes done by this block; the P rows of plane tt are in buffer tt & 1
  float bsg = 0.f, bsg8 = 0.f;  // channels g, g + 8 of P over this warp's share of the chunks (bias gradient)
  unsigned chunk = 0;            // chunks of 16 positions done by this block; chunk % 9 adds its fragments
  // fine rows 2 cy - 1 .. 2 cy + 1 of fine plane f over fine x 2 x0 - 1 .. 2 x0 + 2 seg - 1
  auto stage_fine = [&](int f, int cy, int x0) {
    const uint32_t d = smem_u32(slot(f));
    const bool fin = f >= 0 && f < mq;
    for (int r = 0; r < 3; ++r) {
      const int fy = 2 * cy - 1 + r;
      for (int i = threadIdx.x; i < Wf; i += blockDim.x) {
        const int fx = 2 * x0 - 1 + i;
        const uint4* src = qg;
        uint32_t bytes = 0;
        if (fin && fy >= 0 && fy < mq && fx >= 0 && fx < mq) {
          src = qg + 2 * (fx + (long long)mq * (fy + (long long)mq * f));
          bytes = 16;
        }
        cp_async16(d + (uint32_t)(r * Wf + i) * 16u, src, bytes);
        cp_async16(d + (uint32_t)hs + (uint32_t)(r * Wf + i) * 16u, src + 1, bytes);
      }
    }
  };
  // P rows of coarse voxels (x0 + k, cy, cz), k < seg, zero past the grid
  auto stage_p = [&](int cz, int cy, int x0, unsigned char* buf) {
    const uint32_t d = smem_u32(buf);
    for (int k = threadIdx.x; k < seg; k += blockDim.x) {
      const uint4* src = pg;
      uint32_t bytes = 0;
      if (x0 + k < mp) {
        src = pg + 2 * ((x0 + k) + (long long)mp * (cy + (long long)mp * cz));
        bytes = 16;
      }
      cp_async16(d + (uint32_t)k * 16u, src, bytes);
      cp_async16(d + (uint32_t)(seg + k) * 16u, src + 1, bytes);
    }
  };
  for (long long unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
    const int cy = int(unit % mp);
    const long long rest = unit / mp;
    const int x0 = int(rest % nseg) * seg, zb = int(rest / nseg) * zc, ze = min(mp, zb + zc);
    for (int f = 2 * zb - 1; f <= 2 * zb + 1; ++f) stage_fine(f, cy, x0);
    stage_p(zb, cy, x0, sP0 + (tt & 1u) * 2 * seg * 16);
    asm volatile("cp.async.commit_group;" ::: "memory");
    cp_async_wait_all();
    __syncthreads();
    for (int cz = zb; cz < ze; ++cz, ++tt) {
      if (cz + 1 < ze) {  // fine planes 2 cz + 2, 2 cz + 3 take the slots of 2 cz - 3, 2 cz - 2
        stage_fine(2 * cz + 2, cy, x0);
        stage_fine(2 * cz + 3, cy, x0);
        stage_p(cz + 1, cy, x0, sP0 + ((tt + 1) & 1u) * 2 * seg * 16);
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      const uint32_t sp = smem_u32(sP0 + (tt & 1u) * 2 * seg * 16);
      for (int c = 0; c < seg / 16; ++c) {
        // A = P^T on positions 16c..16c+15: matrices (k 0-7, a lo), (k 0-7, a hi), (k 8-15, a lo), (k 8-15, a hi)
        uint32_t a0, a1, a2, a3;
        ldsm_x4_trans(sp + (uint32_t)(((lm & 1) * seg + 16 * c + (lm >> 1) * 8 + lr) * 16), a0, a1, a2, a3);
        const int k = 16 * c + (lm & 1) * 8 + lr;  // this lane's B row: position k, channel half lm >> 1
#pragma unroll
        for (int jt = 0; jt < 3; ++jt) {
          const int tap = 3 * warp + jt;
          const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
          // B: matrices (k 0-7, b lo), (k 8-15, b lo), (k 0-7, b hi), (k 8-15, b hi)
          uint32_t b0, b1, b2, b3;
          ldsm_x4_trans(smem_u32(slot(2 * cz + dz)) +
                            (uint32_t)((lm >> 1) * hs + ((dy + 1) * Wf + 2 * k + dx + 1) * 16),
                        b0, b1, b2, b3);
          mma16816(acc[jt][0], a0, a1, a2, a3, b0, b1);
          mma16816(acc[jt][1], a0, a1, a2, a3, b2, b3);
        }
        // the bias gradient's share, after the MMAs have consumed the fragment
        if (bpartial && chunk % (kWgThreads / 32) == (unsigned)warp) frag_channel_sums(a0, a1, a2, a3, bsg, bsg8);
        ++chunk;
      }
      cp_async_wait_all();
      __syncthreads();
    }
  }
  if (bpartial) bias_partial_store(bsg, bsg8, bpartial);
  float* out = partial + (long long)blockIdx.x * 27 * 256;
#pragma unroll
  for (int jt = 0; jt < 3; ++jt) {
    const int tap = 3 * warp + jt;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int b = 8 * h + 2 * t;
      out[tap * 256 + g * 16 + b] = acc[jt][h][0];
      out[tap * 256 + g * 16 + b + 1] = acc[jt][h][1];
      out[tap * 256 + (g + 8) * 16 + b] = acc[jt][h][2];
      out[tap * 256 + (g + 8) * 16 + b + 1] = acc[jt][h][3];
    }
  }
}

// Column height z (<= kTcZ output planes per unit) for `slots` resident blocks and `per_slab`
// units per z-slab: fewest plane steps on the slowest block, ceil(units / slots) units of
// `mult` z + `add` steps each (input planes of the column plus about two steps of set-up).
int wave_column(long long per_slab, int m, long long slots, int mult, int add) {
  int zc = 1;
  long long best = -1;
  for (int z = 1; z <= kTcZ; ++z) {
    const long long units = per_slab * ((m + z - 1) / z);
    const long long cost = (units + slots - 1) / slots * (mult * z + add);
    if (best < 0 || cost < best) best = cost, zc = z;
  }
  return zc;
}

// Tiles per block column along z of the transposed convolution, for a grid of m planes with
// per_plane tiles each: kTcZ, or fewer so that a small grid still gives about kTcUnits units.
int tc_column(long long per_plane, int m) {
  return (int)std::max<long long>(1, std::min<long long>(kTcZ, per_plane * m / kTcUnits));
}

void up_tc_launch(const ConvArgs& a, unsigned* status, cudaStream_t s) {
  const size_t smem = up_tc_smem(a.m_in);
  cudaFuncSetAttribute(k_up_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long long mi = a.m_in, per_plane = (mi * (mi + 1) + 127) / 128;
  const int zc = tc_column(per_plane, (int)mi);
  const long long nunits = per_plane * ((mi + zc - 1) / zc);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = 4ll * std::max(nsm, 1);  // 4 blocks per SM (launch bounds, TMEM)
  k_up_tc<<<(int)std::min<long long>(nunits, slots), kTcThreads, smem, s>>>(a, zc, status);
}

typedef CUresult (*TensorMapEncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                         const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                         CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// The driver's tiled tensor-map encoder, looked up once (null if the driver lacks it).
TensorMapEncodeTiled tensor_map_encoder() {
  static const TensorMapEncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (TensorMapEncodeTiled) nullptr;
    return reinterpret_cast<TensorMapEncodeTiled>(p);
  }();
  return fn;
}
__global__ void k_flag(unsigned* status, unsigned bit) { atomicOr(status, bit); }

// A stride-1 convolution: the tensor map of the input (boxes of NY padded rows of one channel
// half), then the streaming kernel on 4 blocks per SM (or fewer if shared memory limits it).
void conv_tc_launch(const ConvArgs& a, unsigned* status, cudaStream_t s) {
  const int m = a.m_out;
  int nstrips = 0;
  const int W = conv_strip_width(m, &nstrips), R = W + 2;
  CUtensorMap map;
  const TensorMapEncodeTiled enc = tensor_map_encoder();
  const cuuint64_t dims[5] = {8, 2, (cuuint64_t)m, (cuuint64_t)m, (cuuint64_t)m};
  const cuuint64_t strides[4] = {16, 32, 32ull * (cuuint64_t)m, 32ull * (cuuint64_t)m * (cuuint64_t)m};
  const cuuint32_t box[5] = {8, 1, (cuuint32_t)R, (cuuint32_t)tma_ny(R), 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (!enc || enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(a.in), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    k_flag<<<1, 1, 0, s>>>(status, kStatusTmaSetup);
    return;
  }
  const size_t smem = conv_tc_smem(m);
  cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  const long long per_plane = ((long long)m * R + 127) / 128;
  int dev = 0, nsm = 0, smem_sm = 0;  // of the current device (attribute queries are cheap)
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = (long long)std::max(1, std::min(4, smem_sm / (int)(smem + 1024))) * std::max(nsm, 1);
  const int zc = wave_column(per_plane * nstrips, m, slots, 1, 4);  // z + 2 planes per column
  const long long nunits = per_plane * nstrips * ((m + zc - 1) / zc);
  k_conv_tc<<<(int)std::min<long long>(nunits, slots), kTcSThreads, smem, s>>>(a, map, zc, W, nstrips, status);
}

// A stride-2 convolution on tcgen05 (k_down_tc): x-strips of at most kDnStripMax coarse
// columns, blocks per SM by shared memory (at most 4, the TMEM budget).
void down_tc_launch(const ConvArgs& a, unsigned* status, cudaStream_t s) {
  const int mo = a.m_out;
  const int nstrips = (mo + kDnStripMax - 1) / kDnStripMax, W = (mo + nstrips - 1) / nstrips;
  const size_t smem = down_tc_smem(W);
  cudaFuncSetAttribute(k_down_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_down_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  const long long per_plane = ((long long)mo * (W + 2) + 127) / 128;
  int dev = 0, nsm = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = (long long)std::max(1, std::min(4, smem_sm / (int)(smem + 1024))) * std::max(nsm, 1);
  const int zc = wave_column(per_plane * nstrips, mo, slots, 2, 3);  // 2 z + 1 planes per column
  const long long nunits = per_plane * nstrips * ((mo + zc - 1) / zc);
  k_down_tc<<<(int)std::min<long long>(nunits, slots), kTcSThreads, smem, s>>>(a, zc, W, nstrips, status);
}

// out = act(conv_G(in; w) + bias + add) * mask
void conv(int gather, const __nv_bfloat16* in, int m_in, const __nv_bfloat16* w, const float* bias,
          const __nv_bfloat16* add, const __nv_bfloat16* mask, bool relu, __nv_bfloat16* out, float* out_planar,
          int m_out, cudaStream_t s, unsigned* status) {
  ConvArgs a{in, m_in, w, bias, add, mask, relu ? 1 : 0, out, out_planar, m_out};
  if (gather == S1)
    conv_tc_launch(a, status, s);
  else if (gather == DOWN2)
    down_tc_launch(a, status, s);
  else
    up_tc_launch(a, status, s);
}

// Weight gradient of `layer`; with bias_from_p also its bias gradient (the channel sums of P,
// the layer's output gradient), from the same kernel.
void wgrad(UNet& u, int layer, int gather, const __nv_bfloat16* P, int mp, const __nv_bfloat16* Q, int mq,
           bool bias_from_p, cudaStream_t s) {
  float* bpart = bias_from_p ? u.partial + (long long)kWgBlocks * 27 * 256 : nullptr;
  int blocks;
  if (gather == S1) {  // stride 1: P and Q on the same grid (mp == mq), in x-strips as k_conv_tc
    int nstrips = 0;
    const int W = conv_strip_width(mp, &nstrips);
    const size_t smem = wgrad_s1_smem(W);
    cudaFuncSetAttribute(k_wgrad_s1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const long long per_plane = ((long long)mp * (W + 2) + 127) / 128;
    const int zc = wave_column(per_plane * nstrips, mp, kWgBlocks, 1, 4);
    blocks = (int)std::min<long long>(kWgBlocks, per_plane * nstrips * ((mp + zc - 1) / zc));
    k_wgrad_s1<<<blocks, kWgThreads, smem, s>>>(P, Q, mp, zc, W, nstrips, u.partial, bpart);
  } else {  // stride 2: P on the coarse grid, Q on the fine grid
    int nseg = 0;
    const int seg = wgrad_s2_seg(mp, &nseg);
    const size_t smem = wgrad_s2_smem(seg);
    cudaFuncSetAttribute(k_wgrad_s2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const long long per_plane = (long long)mp * nseg;
    const int zc = (int)std::max<long long>(1, std::min<long long>(kTcZ, per_plane * mp / kTcUnits));
    blocks = (int)std::min<long long>(kWgBlocks, per_plane * ((mp + zc - 1) / zc));
    k_wgrad_s2<<<blocks, kWgThreads, smem, s>>>(P, mp, Q, mq, seg, nseg, zc, u.partial, bpart);
  }
  const UNetLayer& L = u.L[layer];
  k_wgrad_reduce<<<27 * 256 / 32 + (bias_from_p ? 1 : 0), 1024, 0, s>>>(
      u.partial, bpart, blocks, u.grads + L.woff, bias_from_p ? u.grads + L.boff : nullptr, L.kind, L.cin, L.cout);
}

void bgrad(UNet& u, int layer, const __nv_bfloat16* P, long long nvox, cudaStream_t s) {
  const int blocks = (int)std::min<long long>(kBgBlocks, (nvox + 255) / 256);
  float* part = u.partial + (long long)kWgBlocks * 27 * 256;
  k_bgrad_partial<<<blocks, 256, 0, s>>>(P, nvox, part);
  k_bgrad_reduce<<<1, 256, 0, s>>>(part, blocks, u.grads + u.L[layer].boff, u.L[layer].cout);
}

}  // namespace

// ------------------------------------------------------------------ host API pieces
nhmf_status unet_alloc(nhmf_ctx* c, int cap) {
  if ((c->g.M - 1) % 4 != 0) return fail(c, NHMF_ERR_ARG, "unet: p*N must be divisible by 4 (two stride-2 levels)");
  // the stride-1 tensor-core convolution stages a ring of padded planes of the finest grid in
  // shared memory: 27 * 512 + 8 (130 + 2 (M + 2)) 16 + 16 bytes <= 227 KB
  if (c->g.M > 785) return fail(c, NHMF_ERR_ARG, "unet: at most 785 nodes per direction (p*N <= 784)");
  if (c->unet) return fail(c, NHMF_ERR_STATE, "unet: already created");
  UNet* u = new UNet();
  c->unet = u;
  u->status = c->status;
  u->M0 = c->g.M;
  u->M1 = (u->M0 - 1) / 2 + 1;
  u->M2 = (u->M1 - 1) / 2 + 1;
  u->N0 = (long long)u->M0 * u->M0 * u->M0;
  u->N1 = (long long)u->M1 * u->M1 * u->M1;
  u->N2 = (long long)u->M2 * u->M2 * u->M2;
  long long off = 0;
  for (int l = 0; l < 11; ++l) {
    UNetLayer& L = u->L[l];
    L.kind = kLayerKind[l];
    L.cin = kLayerCin[l];
    L.cout = kLayerCout[l];
    L.woff = off;
    off += (long long)L.cin * L.cout * 27;
    L.boff = off;
    off += L.cout;
  }
  u->nparams = off;
  u->cap = cap;
  bool ok = true;
  auto A = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
    if (ok) cudaMemset(*p, 0, bytes);
  };
  A((void**)&u->params, off * sizeof(float));
  A((void**)&u->grads, off * sizeof(float));
  A((void**)&u->adam_m, off * sizeof(float));
  A((void**)&u->adam_v, off * sizeof(float));
  for (int l = 0; l < 11; ++l) {
    A((void**)&u->L[l].wf, 27 * 256 * sizeof(__nv_bfloat16));
    A((void**)&u->L[l].wb, 27 * 256 * sizeof(__nv_bfloat16));
  }
  const size_t b0 = u->N0 * kC * sizeof(__nv_bfloat16), b1 = u->N1 * kC * sizeof(__nv_bfloat16),
               b2 = u->N2 * kC * sizeof(__nv_bfloat16);
  for (__nv_bfloat16** p : {&u->x16, &u->a0, &u->s0, &u->u0, &u->t0, &u->g0a, &u->g0b, &u->g0c}) A((void**)p, b0);
  for (__nv_bfloat16** p : {&u->d1, &u->s1, &u->u1, &u->t1, &u->g1a, &u->g1b, &u->g1c}) A((void**)p, b1);
  for (__nv_bfloat16** p : {&u->d2, &u->m2, &u->g2a, &u->g2b}) A((void**)p, b2);
  A((void**)&u->y, 3 * u->N0 * sizeof(float));
  A((void**)&u->partial, ((size_t)kWgBlocks * 27 * 256 + (size_t)kBgBlocks * 16) * sizeof(float));
  A((void**)&u->sc, 16 * sizeof(double));
  if (cap > 0) A((void**)&u->pairs, (size_t)cap * 2 * 3 * u->N0 * sizeof(float));
  if (!ok) return fail(c, NHMF_ERR_OOM, "unet: device allocation failed");
  return NHMF_OK;
}

void unet_free(nhmf_ctx* c) {
  UNet* u = c->unet;
  if (!u) return;
  void* ptrs[] = {u->params, u->grads, u->adam_m, u->adam_v, u->x16, u->a0, u->s0, u->d1, u->s1, u->d2, u->m2,
                  u->u1, u->t1, u->u0, u->t0, u->g0a, u->g0b, u->g0c, u->g1a, u->g1b, u->g1c, u->g2a, u->g2b,
                  u->y, u->partial, u->sc, u->pairs};
  for (void* p : ptrs) cudaFree(p);
  for (int l = 0; l < 11; ++l) {
    cudaFree(u->L[l].wf);
    cudaFree(u->L[l].wb);
  }
  delete u;
  c->unet = nullptr;
}

void unet_refresh_weights(UNet& u, cudaStream_t s) {
  for (int l = 0; l < 11; ++l) {
    const UNetLayer& L = u.L[l];
    k_layer_weights<<<(27 * 256 + 255) / 256, 256, 0, s>>>(u.params + L.woff, L.kind, L.cin, L.cout, L.wf, L.wb);
  }
}

// Forward pass from u.x16 to u.y (FP32 planar).
void unet_forward(UNet& u, cudaStream_t s) {
  const float* P = u.params;
  auto B = [&](int l) { return P + u.L[l].boff; };
  const int M0 = u.M0, M1 = u.M1, M2 = u.M2;
  conv(S1, u.x16, M0, u.L[L_IN].wf, B(L_IN), nullptr, nullptr, true, u.a0, nullptr, M0, s, u.status);
  conv(S1, u.a0, M0, u.L[L_E0].wf, B(L_E0), nullptr, nullptr, true, u.s0, nullptr, M0, s, u.status);
  conv(DOWN2, u.s0, M0, u.L[L_D1].wf, B(L_D1), nullptr, nullptr, true, u.d1, nullptr, M1, s, u.status);
  conv(S1, u.d1, M1, u.L[L_E1].wf, B(L_E1), nullptr, nullptr, true, u.s1, nullptr, M1, s, u.status);
  conv(DOWN2, u.s1, M1, u.L[L_D2].wf, B(L_D2), nullptr, nullptr, true, u.d2, nullptr, M2, s, u.status);
  conv(S1, u.d2, M2, u.L[L_M2].wf, B(L_M2), nullptr, nullptr, true, u.m2, nullptr, M2, s, u.status);
  conv(UP2, u.m2, M2, u.L[L_U1].wf, B(L_U1), u.s1, nullptr, true, u.u1, nullptr, M1, s, u.status);
  conv(S1, u.u1, M1, u.L[L_T1].wf, B(L_T1), nullptr, nullptr, true, u.t1, nullptr, M1, s, u.status);
  conv(UP2, u.t1, M1, u.L[L_U0].wf, B(L_U0), u.s0, nullptr, true, u.u0, nullptr, M0, s, u.status);
  conv(S1, u.u0, M0, u.L[L_T0].wf, B(L_T0), nullptr, nullptr, true, u.t0, nullptr, M0, s, u.status);
  conv(S1, u.t0, M0, u.L[L_OUT].wf, B(L_OUT), nullptr, nullptr, false, nullptr, u.y, M0, s, u.status);
}

// Backward pass from dy16 (in u.g0a) to u.grads (after unet_forward on the same input).
void unet_backward(UNet& u, cudaStream_t s) {
  const int M0 = u.M0, M1 = u.M1, M2 = u.M2;
  __nv_bfloat16 *dy = u.g0a, *dt0 = u.g0b, *du0 = u.g0c, *ds0 = u.g0a;
  __nv_bfloat16 *dt1 = u.g1a, *du1 = u.g1b, *ds1 = u.g1c, *dd1 = u.g1a;
  __nv_bfloat16 *dm2 = u.g2a, *dd2 = u.g2b;
  wgrad(u, L_OUT, S1, dy, M0, u.t0, M0, true, s);
  conv(S1, dy, M0, u.L[L_OUT].wb, nullptr, nullptr, u.t0, false, dt0, nullptr, M0, s, u.status);
  wgrad(u, L_T0, S1, dt0, M0, u.u0, M0, true, s);
  conv(S1, dt0, M0, u.L[L_T0].wb, nullptr, nullptr, u.u0, false, du0, nullptr, M0, s, u.status);
  wgrad(u, L_U0, DOWN2, u.t1, M1, du0, M0, false, s);  // dU[c][o] = sum t1[c] du0[o](2v'+d)
  bgrad(u, L_U0, du0, u.N0, s);
  conv(DOWN2, du0, M0, u.L[L_U0].wb, nullptr, nullptr, u.t1, false, dt1, nullptr, M1, s, u.status);
  wgrad(u, L_T1, S1, dt1, M1, u.u1, M1, true, s);
  conv(S1, dt1, M1, u.L[L_T1].wb, nullptr, nullptr, u.u1, false, du1, nullptr, M1, s, u.status);
  wgrad(u, L_U1, DOWN2, u.m2, M2, du1, M1, false, s);
  bgrad(u, L_U1, du1, u.N1, s);
  conv(DOWN2, du1, M1, u.L[L_U1].wb, nullptr, nullptr, u.m2, false, dm2, nullptr, M2, s, u.status);
  wgrad(u, L_M2, S1, dm2, M2, u.d2, M2, true, s);
  conv(S1, dm2, M2, u.L[L_M2].wb, nullptr, nullptr, u.d2, false, dd2, nullptr, M2, s, u.status);
  wgrad(u, L_D2, DOWN2, dd2, M2, u.s1, M1, true, s);
  conv(UP2, dd2, M2, u.L[L_D2].wb, nullptr, du1, u.s1, false, ds1, nullptr, M1, s, u.status);  // + skip grad, ReLU mask
  wgrad(u, L_E1, S1, ds1, M1, u.d1, M1, true, s);
  conv(S1, ds1, M1, u.L[L_E1].wb, nullptr, nullptr, u.d1, false, dd1, nullptr, M1, s, u.status);
  wgrad(u, L_D1, DOWN2, dd1, M1, u.s0, M0, true, s);
  conv(UP2, dd1, M1, u.L[L_D1].wb, nullptr, du0, u.s0, false, ds0, nullptr, M0, s, u.status);
  wgrad(u, L_E0, S1, ds0, M0, u.a0, M0, true, s);
  conv(S1, ds0, M0, u.L[L_E0].wb, nullptr, nullptr, u.a0, false, dt0, nullptr, M0, s, u.status);  // da0 in dt0's buffer
  wgrad(u, L_IN, S1, dt0, M0, u.x16, M0, true, s);
}

// x16 from an FP64 planar vector scaled to unit RMS.
void unet_input_from(nhmf_ctx* c, const double* r, cudaStream_t s) {
  UNet& u = *c->unet;
  norm2(3 * u.N0, r, u.sc + 0, c->work ? c->work->partials : nullptr, s);
  k_input<double><<<kConvBlocks, 256, 0, s>>>(r, u.N0, u.sc + 0, std::sqrt(3.0 * u.N0), u.x16);
}

void unet_input_planar32(UNet& u, const float* x, cudaStream_t s) {
  k_input<float><<<kConvBlocks, 256, 0, s>>>(x, u.N0, nullptr, 1.0, u.x16);
}

// Loss of u.y against the FP32 planar target; writes dy16 into u.g0a; adds the loss to
// sc[3] when accumulate is set.  Uses the solver's reduction scratch.
void unet_loss_and_grad(nhmf_ctx* c, const float* target, bool accumulate, cudaStream_t s) {
  UNet& u = *c->unet;
  double* partials = c->work->partials;
  k_loss_partials<<<kRedBlocks, kRedThreads, 0, s>>>(u.y, target, u.N0, c->prm.bc, u.M0, partials);
  k_loss_final<<<1, kRedThreads, 0, s>>>(partials, u.sc + 1, u.sc + 2, accumulate ? u.sc + 3 : nullptr);
  k_loss_grad<<<kConvBlocks, 256, 0, s>>>(u.y, target, u.N0, c->prm.bc, u.M0, u.sc + 2, u.g0a);
}

void unet_adam(UNet& u, float lr, cudaStream_t s) {
  u.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - std::pow(b1, (float)u.step), bc2 = 1.f - std::pow(b2, (float)u.step);
  k_adam<<<256, 256, 0, s>>>(u.nparams, u.params, u.grads, u.adam_m, u.adam_v, lr, b1, b2, 1e-8f, bc1, bc2);
  unet_refresh_weights(u, s);
}

// z = preconditioner(r): network on r scaled to unit RMS, output scaled back by ||r|| / sqrt(3N),
// zero on constrained DoFs.
void unet_precondition(nhmf_ctx* c, const double* r, double* z, cudaStream_t s) {
  UNet& u = *c->unet;
  unet_input_from(c, r, s);
  unet_forward(u, s);
  k_output<<<kConvBlocks, 256, 0, s>>>(u.y, u.N0, c->prm.bc, u.M0, u.sc + 0, 1.0 / std::sqrt(3.0 * u.N0), z);
}

nhmf_status unet_record(nhmf_ctx* c, const double* r, const double* e, cudaStream_t s) {
  UNet& u = *c->unet;
  if (u.npairs >= u.cap) return NHMF_OK;  // store full: later pairs are dropped
  float* slot = u.pairs + (size_t)u.npairs * 2 * 3 * u.N0;
  const double mul = std::sqrt(3.0 * u.N0);
  norm2(3 * u.N0, r, u.sc + 4, c->work->partials, s);
  k_store_scaled<<<kConvBlocks, 256, 0, s>>>(r, 3 * u.N0, u.sc + 4, mul, slot);
  norm2(3 * u.N0, e, u.sc + 5, c->work->partials, s);
  k_store_scaled<<<kConvBlocks, 256, 0, s>>>(e, 3 * u.N0, u.sc + 5, mul, slot + 3 * u.N0);
  u.npairs += 1;
  return cuda_check(c, cudaGetLastError(), "unet record");
}

namespace {
__global__ void k_store_f32(const double* src, long long n3, float* dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    dst[i] = float(src[i]);
}
// dst = (float(xstar) - dst) * mul / ||float(xstar) - dst|| in two passes
__global__ void k_sub_from(const double* xstar, long long n3, float* dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    dst[i] = float(xstar[i] - double(dst[i]));
}
__global__ void k_scale_f32(long long n3, const double* nrm, double mul, float* dst) {
  const float s = float(*nrm > 0.0 ? mul / *nrm : 0.0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    dst[i] *= s;
}
}  // namespace

namespace {
// splitmix64 (Steele, Lea and Flood 2014): output k of seed s is mix(s + (k + 1) * gamma).
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// standard normal from outputs 2k and 2k+1 (Box-Muller, first of the pair)
__device__ __forceinline__ double normal_at(unsigned long long seed, unsigned long long k) {
  const double u1 = 1.0 - double(splitmix64_at(seed, 2 * k) >> 11) * 0x1.0p-53;
  const double u2 = double(splitmix64_at(seed, 2 * k + 1) >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}
// Random field at one lattice scale: e_c(x) = trilinear interpolant of N(0,1) values on a
// (2^L + 1)^3 lattice over the unit cube (node coordinates i/(M-1)); L = 1 + seed mod Lmax with
// 2^Lmax = M - 1, so the pairs of consecutive seeds sweep from the coarsest lattice to nodal
// white noise.  Zero on constrained DoFs.
__global__ void k_smooth_field(double* e, int M, int bc, unsigned long long seed) {
  const long long n = (long long)M * M * M;
  int Lmax = 0;
  while ((1 << (Lmax + 1)) <= M - 1) ++Lmax;
  const int L = 1 + int(seed % (unsigned long long)Lmax);
  const int G = (1 << L) + 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * n; i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i / n);
    const long long v = i % n;
    const int x = int(v % M), y = int((v / M) % M), z = int(v / ((long long)M * M));
    if (constrained_dof(bc, c, v, M)) {
      e[i] = 0.0;
      continue;
    }
    const double fx = double(x) / (M - 1) * (G - 1), fy = double(y) / (M - 1) * (G - 1), fz = double(z) / (M - 1) * (G - 1);
    const int ix = min(int(fx), G - 2), iy = min(int(fy), G - 2), iz = min(int(fz), G - 2);
    const double tx = fx - ix, ty = fy - iy, tz = fz - iz;
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const unsigned long long k = (unsigned long long)c * G * G * G + (ix + dx) + (unsigned long long)G * ((iy + dy) + G * (iz + dz));
          const double wgt = (dx ? tx : 1.0 - tx) * (dy ? ty : 1.0 - ty) * (dz ? tz : 1.0 - tz);
          acc += wgt * normal_at(seed, k);
        }
    e[i] = acc;
  }
}
}  // namespace

void unet_smooth_field(nhmf_ctx* c, double* e, unsigned long long seed, cudaStream_t s) {
  k_smooth_field<<<kConvBlocks, 256, 0, s>>>(e, c->g.M, c->prm.bc, seed);
}

// CG snapshot: input slot <- r_j normalised, target slot <- x_j (finished later).
int unet_snapshot_begin(nhmf_ctx* c, const double* r, const double* xj, cudaStream_t s) {
  UNet& u = *c->unet;
  if (u.npairs >= u.cap) return -1;
  const int slot = u.npairs++;
  float* p = u.pairs + (size_t)slot * 2 * 3 * u.N0;
  norm2(3 * u.N0, r, u.sc + 4, c->work->partials, s);
  k_store_scaled<<<kConvBlocks, 256, 0, s>>>(r, 3 * u.N0, u.sc + 4, std::sqrt(3.0 * u.N0), p);
  k_store_f32<<<kConvBlocks, 256, 0, s>>>(xj, 3 * u.N0, p + 3 * u.N0);
  return slot;
}

// target slot <- (x* - x_j) normalised to unit RMS.
void unet_snapshot_finish(nhmf_ctx* c, int slot, const double* xstar, cudaStream_t s) {
  UNet& u = *c->unet;
  float* tgt = u.pairs + (size_t)slot * 2 * 3 * u.N0 + 3 * u.N0;
  k_sub_from<<<kConvBlocks, 256, 0, s>>>(xstar, 3 * u.N0, tgt);
  norm2(3 * u.N0, tgt, u.sc + 5, c->work->partials, s);
  k_scale_f32<<<kConvBlocks, 256, 0, s>>>(3 * u.N0, u.sc + 5, std::sqrt(3.0 * u.N0), tgt);
}

}  // namespace nhmf

// ------------------------------------------------------------------ C ABI
using namespace nhmf;

extern "C" {

nhmf_status nhmf_unet_create(nhmf_ctx* c, int pair_capacity) {
  if (!c) return NHMF_ERR_ARG;
  if (pair_capacity < 0) return fail(c, NHMF_ERR_ARG, "unet_create: negative capacity");
  nhmf_status st = ensure_work(c);
  if (st != NHMF_OK) return st;
  st = unet_alloc(c, pair_capacity);
  if (st != NHMF_OK) {
    unet_free(c);
    return st;
  }
  return cuda_check(c, cudaDeviceSynchronize(), "unet_create");
}

size_t nhmf_unet_num_params(const nhmf_ctx* c) { return (c && c->unet) ? (size_t)c->unet->nparams : 0; }

int nhmf_unet_num_pairs(const nhmf_ctx* c) { return (c && c->unet) ? c->unet->npairs : 0; }

nhmf_status nhmf_unet_set_params(nhmf_ctx* c, const float* host, size_t n) {
  if (!c) return NHMF_ERR_ARG;
  if (!c->unet) return fail(c, NHMF_ERR_STATE, "unet_set_params: no network");
  UNet& u = *c->unet;
  if (!host || n != (size_t)u.nparams) return fail(c, NHMF_ERR_ARG, "unet_set_params: size mismatch");
  nhmf_status st = cuda_check(c, cudaMemcpy(u.params, host, n * sizeof(float), cudaMemcpyHostToDevice), "params copy");
  if (st != NHMF_OK) return st;
  cudaMemset(u.adam_m, 0, n * sizeof(float));
  cudaMemset(u.adam_v, 0, n * sizeof(float));
  u.step = 0;
  unet_refresh_weights(u, 0);
  return cuda_check(c, cudaDeviceSynchronize(), "unet_set_params");
}

nhmf_status nhmf_unet_get_params(nhmf_ctx* c, float* host, size_t n) {
  if (!c) return NHMF_ERR_ARG;
  if (!c->unet) return fail(c, NHMF_ERR_STATE, "unet_get_params: no network");
  if (!host || n != (size_t)c->unet->nparams) return fail(c, NHMF_ERR_ARG, "unet_get_params: size mismatch");
  return cuda_check(c, cudaMemcpy(host, c->unet->params, n * sizeof(float), cudaMemcpyDeviceToHost), "params read");
}

nhmf_status nhmf_unet_forward(nhmf_ctx* c, const float* x, float* y, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!c->unet) return fail(c, NHMF_ERR_STATE, "unet_forward: no network");
  if (!x || !y) return fail(c, NHMF_ERR_ARG, "unet_forward: bad argument");
  UNet& u = *c->unet;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unet_input_planar32(u, x, s);
  unet_forward(u, s);
  return cuda_check(c, cudaMemcpyAsync(y, u.y, 3 * u.N0 * sizeof(float), cudaMemcpyDeviceToDevice, s), "unet_forward");
}

nhmf_status nhmf_unet_loss_grad(nhmf_ctx* c, const float* x, const float* e, double* loss, float* grads_host,
                                void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!c->unet) return fail(c, NHMF_ERR_STATE, "unet_loss_grad: no network");
  if (!x || !e || !loss) return fail(c, NHMF_ERR_ARG, "unet_loss_grad: bad argument");
  UNet& u = *c->unet;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unet_input_planar32(u, x, s);
  unet_forward(u, s);
  unet_loss_and_grad(c, e, false, s);
  unet_backward(u, s);
  double nd[2];
  nhmf_status st = cuda_check(c, cudaMemcpyAsync(nd, u.sc + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), "loss read");
  if (st == NHMF_OK && grads_host)
    st = cuda_check(c, cudaMemcpyAsync(grads_host, u.grads, u.nparams * sizeof(float), cudaMemcpyDeviceToHost, s), "grad read");
  if (st == NHMF_OK) st = cuda_check(c, cudaStreamSynchronize(s), "loss_grad sync");
  if (st == NHMF_OK) st = nhmf_check_status(c, stream);  // tensor-core waits and tensor maps
  *loss = nd[1] > 0.0 ? nd[0] / nd[1] : 0.0;
  return st;
}

nhmf_status nhmf_unet_precondition(nhmf_ctx* c, const double* r, double* z, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!c->unet) return fail(c, NHMF_ERR_STATE, "unet_precondition: no network");
  if (!r || !z) return fail(c, NHMF_ERR_ARG, "unet_precondition: bad argument");
  unet_precondition(c, r, z, static_cast<cudaStream_t>(stream));
  return cuda_check(c, cudaGetLastError(), "unet_precondition");
}

nhmf_status nhmf_unet_record_pair(nhmf_ctx* c, const double* r, const double* e, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!c->unet) return fail(c, NHMF_ERR_STATE, "unet_record_pair: no network");
  if (!r || !e) return fail(c, NHMF_ERR_ARG, "unet_record_pair: bad argument");
  return unet_record(c, r, e, static_cast<cudaStream_t>(stream));
}

nhmf_status nhmf_unet_train(nhmf_ctx* c, int epochs, double lr, double* loss_first, double* loss_last, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!c->unet) return fail(c, NHMF_ERR_STATE, "unet_train: no network");
  if (epochs < 1 || !(lr > 0.0) || !loss_first || !loss_last) return fail(c, NHMF_ERR_ARG, "unet_train: bad argument");
  UNet& u = *c->unet;
  if (u.npairs == 0) return fail(c, NHMF_ERR_STATE, "unet_train: no recorded pairs");
  NvtxRange range("nhmf_unet_train");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t pair_stride = (size_t)2 * 3 * u.N0;
  for (int ep = 0; ep < epochs; ++ep) {
    cudaMemsetAsync(u.sc + 3, 0, sizeof(double), s);
    for (int k = 0; k < u.npairs; ++k) {
      const float* slot = u.pairs + (size_t)k * pair_stride;
      unet_input_planar32(u, slot, s);
      unet_forward(u, s);
      unet_loss_and_grad(c, slot + 3 * u.N0, true, s);
      unet_backward(u, s);
      unet_adam(u, (float)lr, s);
    }
    double acc = 0.0;
    nhmf_status st = cuda_check(c, cudaMemcpyAsync(&acc, u.sc + 3, sizeof(double), cudaMemcpyDeviceToHost, s), "train loss");
    if (st == NHMF_OK) st = cuda_check(c, cudaStreamSynchronize(s), "train sync");
    if (st == NHMF_OK) st = nhmf_check_status(c, stream);  // tensor-core waits and tensor maps
    if (st != NHMF_OK) return st;
    if (!std::isfinite(acc)) return fail(c, NHMF_ERR_NONFINITE, "unet_train: non-finite loss");
    if (ep == 0) *loss_first = acc / u.npairs;
    *loss_last = acc / u.npairs;
  }
  return NHMF_OK;
}

}  // extern "C"
