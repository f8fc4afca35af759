// Vector kernels of the Krylov solvers (Section 2.3: CG on the matrix-free operator).
// Reductions are deterministic: a fixed grid of kRedBlocks blocks accumulates FP64 partial
// sums with a fixed grid-stride order and a fixed shuffle tree; one block then reduces the
// partials in a fixed order.  Results stay on the device.
#include "blas.h"

namespace nhmf {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NS accumulators and write partials[s * kRedBlocks + blockIdx.x].
template <int NS>
__device__ __forceinline__ void block_partials(double (&acc)[NS], double* partials) {
  __shared__ double sh[NS][kRedThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double v = warp_sum(acc[s]);
    if (lane == 0) sh[s][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double v = lane < kRedThreads / 32 ? sh[s][lane] : 0.0;
      v = warp_sum(v);
      if (lane == 0) partials[s * kRedBlocks + blockIdx.x] = v;
    }
  }
}

// out[s] = sum over partials of slot s; one block of kRedThreads threads.
__global__ void k_final(const double* partials, int ns, double* out0, double* out1, double* out2) {
  __shared__ double sh[kRedThreads / 32];
  double* outs[3] = {out0, out1, out2};
  for (int s = 0; s < ns; ++s) {
    double v = 0.0;
    for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) v += partials[s * kRedBlocks + i];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      double w = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
      w = warp_sum(w);
      if (threadIdx.x == 0 && outs[s]) *outs[s] = w;
    }
    __syncthreads();
  }
}

template <typename TX, typename TY>
__global__ void __launch_bounds__(kRedThreads) k_dot(long long n, const TX* x, const TY* y, double* partials) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads)
    acc[0] = fma(double(x[i]), double(y[i]), acc[0]);
  block_partials<1>(acc, partials);
}

// PCG update (Jacobi): alpha = rz/pq; x += alpha p; r -= alpha q; z = dinv r;
// partial sums of r.z and r.r.  A non-positive p.q is a breakdown: alpha = 0 and flag.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_pcg_update(long long n, const double* rz, const double* pq, T* x, T* r,
                                                            const T* p, const T* q, const T* dinv, T* z,
                                                            double* partials, unsigned* flag) {
  const double pqv = *pq;
  const bool ok = pqv > 0.0 && isfinite(pqv);
  const T alpha = ok ? T(*rz / pqv) : T(0);
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flag, 4u);
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads) {
    x[i] = fma(alpha, p[i], x[i]);
    const T ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    const T zi = dinv[i] * ri;
    z[i] = zi;
    acc[0] = fma(double(ri), double(zi), acc[0]);
    acc[1] = fma(double(ri), double(ri), acc[1]);
  }
  block_partials<2>(acc, partials);
}

// p = z + beta p with beta = rz_new / rz_old (beta = 0 when rz_old is null).
template <typename T>
__global__ void k_pcg_direction(long long n, const double* rz_new, const double* rz_old, const T* z, T* p) {
  const T beta = rz_old ? T(*rz_new / *rz_old) : T(0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = rz_old ? fma(beta, p[i], z[i]) : z[i];
}

// z = dinv r and partial sums of r.z, r.r (start of PCG).
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_jacobi(long long n, const T* r, const T* dinv, T* z, double* partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads) {
    const T zi = dinv[i] * r[i];
    z[i] = zi;
    acc[0] = fma(double(r[i]), double(zi), acc[0]);
    acc[1] = fma(double(r[i]), double(r[i]), acc[1]);
  }
  block_partials<2>(acc, partials);
}

// y = a x + b y with scalars a = sa * (*pa) (pa may be null -> sa), same for b.
__global__ void k_axpby(long long n, double sa, const double* pa, const double* x, double sb, const double* pb, double* y) {
  const double a = pa ? sa * *pa : sa;
  const double b = pb ? sb * *pb : sb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : fma(a, x[i], b * y[i]);
}

// out = num / den (device scalars), with a sign.
__global__ void k_noise(long long n, double* z, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long v = (unsigned long long)i + seed * 0x9E3779B97F4A7C15ull;
    v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
    v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
    v ^= v >> 31;
    z[i] = double(v >> 11) * 0x1.0p-52 - 1.0;
  }
}

__global__ void k_ratio(const double* num, const double* den, double sign, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = sign * (*num / *den);
}

__global__ void k_ratio_or_zero(const double* num, const double* den, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double r = *num / *den;
    *out = (*den > 0.0 && isfinite(r)) ? r : 0.0;
  }
}

template <typename TI, typename TO>
__global__ void k_scale_convert(long long n, const TI* x, const double* scale, bool invert, TO* y) {
  double s = scale ? *scale : 1.0;
  if (invert) s = s > 0.0 ? 1.0 / s : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = TO(double(x[i]) * s);
}

__global__ void k_reciprocal(long long n, const double* d, double* dinv64, float* dinv32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = 1.0 / d[i];
    if (dinv64) dinv64[i] = v;
    if (dinv32) dinv32[i] = float(v);
  }
}

__global__ void k_mul(long long n, const double* d, double* x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] *= d[i];
}

__global__ void k_sqrt(double* x) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *x = sqrt(*x);
}

constexpr int kEwBlocks = 1216;  // 8 blocks per SM for element-wise kernels
constexpr int kEwThreads = 256;

}  // namespace

void dot(long long n, const double* x, const double* y, double* out, double* partials, cudaStream_t s) {
  k_dot<<<kRedBlocks, kRedThreads, 0, s>>>(n, x, y, partials);
  k_final<<<1, kRedThreads, 0, s>>>(partials, 1, out, nullptr, nullptr);
}
void dot(long long n, const float* x, const float* y, double* out, double* partials, cudaStream_t s) {
  k_dot<<<kRedBlocks, kRedThreads, 0, s>>>(n, x, y, partials);
  k_final<<<1, kRedThreads, 0, s>>>(partials, 1, out, nullptr, nullptr);
}
void norm2(long long n, const double* x, double* out, double* partials, cudaStream_t s) {
  dot(n, x, x, out, partials, s);
  k_sqrt<<<1, 32, 0, s>>>(out);
}
void norm2(long long n, const float* x, double* out, double* partials, cudaStream_t s) {
  dot(n, x, x, out, partials, s);
  k_sqrt<<<1, 32, 0, s>>>(out);
}

template <typename T>
void pcg_update(long long n, const double* rz, const double* pq, T* x, T* r, const T* p, const T* q, const T* dinv, T* z,
                double* rz_new, double* rr, double* partials, unsigned* flag, cudaStream_t s) {
  k_pcg_update<T><<<kRedBlocks, kRedThreads, 0, s>>>(n, rz, pq, x, r, p, q, dinv, z, partials, flag);
  k_final<<<1, kRedThreads, 0, s>>>(partials, 2, rz_new, rr, nullptr);
}
template <typename T>
void pcg_direction(long long n, const double* rz_new, const double* rz_old, const T* z, T* p, cudaStream_t s) {
  k_pcg_direction<T><<<kEwBlocks, kEwThreads, 0, s>>>(n, rz_new, rz_old, z, p);
}
template <typename T>
void jacobi(long long n, const T* r, const T* dinv, T* z, double* rz, double* rr, double* partials, cudaStream_t s) {
  k_jacobi<T><<<kRedBlocks, kRedThreads, 0, s>>>(n, r, dinv, z, partials);
  k_final<<<1, kRedThreads, 0, s>>>(partials, 2, rz, rr, nullptr);
}
template void pcg_update<double>(long long, const double*, const double*, double*, double*, const double*, const double*,
                                 const double*, double*, double*, double*, double*, unsigned*, cudaStream_t);
template void pcg_update<float>(long long, const double*, const double*, float*, float*, const float*, const float*,
                                const float*, float*, double*, double*, double*, unsigned*, cudaStream_t);
template void pcg_direction<double>(long long, const double*, const double*, const double*, double*, cudaStream_t);
template void pcg_direction<float>(long long, const double*, const double*, const float*, float*, cudaStream_t);
template void jacobi<double>(long long, const double*, const double*, double*, double*, double*, double*, cudaStream_t);
template void jacobi<float>(long long, const float*, const float*, float*, double*, double*, double*, cudaStream_t);

void axpby(long long n, double a, const double* pa, const double* x, double b, const double* pb, double* y, cudaStream_t s) {
  k_axpby<<<kEwBlocks, kEwThreads, 0, s>>>(n, a, pa, x, b, pb, y);
}
void ratio(const double* num, const double* den, double sign, double* out, cudaStream_t s) {
  k_ratio<<<1, 32, 0, s>>>(num, den, sign, out);
}
void fill_noise(long long n, double* z, unsigned long long seed, cudaStream_t s) {
  k_noise<<<kRedBlocks, kRedThreads, 0, s>>>(n, z, seed);
}
void ratio_or_zero(const double* num, const double* den, double* out, cudaStream_t s) {
  k_ratio_or_zero<<<1, 32, 0, s>>>(num, den, out);
}
void to_fp32_scaled(long long n, const double* x, const double* scale, bool invert, float* y, cudaStream_t s) {
  k_scale_convert<double, float><<<kEwBlocks, kEwThreads, 0, s>>>(n, x, scale, invert, y);
}
void to_fp64_scaled(long long n, const float* x, const double* scale, double* y, cudaStream_t s) {
  k_scale_convert<float, double><<<kEwBlocks, kEwThreads, 0, s>>>(n, x, scale, false, y);
}
void jacobi_apply(long long n, const double* dinv, double* x, cudaStream_t s) {
  k_mul<<<kEwBlocks, kEwThreads, 0, s>>>(n, dinv, x);
}
void reciprocal(long long n, const double* d, double* dinv64, float* dinv32, cudaStream_t s) {
  k_reciprocal<<<kEwBlocks, kEwThreads, 0, s>>>(n, d, dinv64, dinv32);
}

}  // namespace nhmf
