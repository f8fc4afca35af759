// Vector kernels of the Krylov solvers; scalars live on the device.
#pragma once
#include <cuda_runtime.h>

namespace nhmf {

constexpr int kRedBlocks = 1024;   // fixed reduction grid: results do not depend on timing
constexpr int kRedThreads = 256;
constexpr int kPartialSlots = 3 * kRedBlocks;  // scratch doubles a reduction needs

void dot(long long n, const double* x, const double* y, double* out, double* partials, cudaStream_t s);
void dot(long long n, const float* x, const float* y, double* out, double* partials, cudaStream_t s);
void norm2(long long n, const double* x, double* out, double* partials, cudaStream_t s);
void norm2(long long n, const float* x, double* out, double* partials, cudaStream_t s);
template <typename T>
void pcg_update(long long n, const double* rz, const double* pq, T* x, T* r, const T* p, const T* q, const T* dinv, T* z,
                double* rz_new, double* rr, double* partials, unsigned* flag, cudaStream_t s);
template <typename T>
void pcg_direction(long long n, const double* rz_new, const double* rz_old, const T* z, T* p, cudaStream_t s);
template <typename T>
void jacobi(long long n, const T* r, const T* dinv, T* z, double* rz, double* rr, double* partials, cudaStream_t s);
void axpby(long long n, double a, const double* pa, const double* x, double b, const double* pb, double* y, cudaStream_t s);
void ratio(const double* num, const double* den, double sign, double* out, cudaStream_t s);
// out = num / den if den > 0 and the quotient is finite, else 0 (a guarded step length)
void ratio_or_zero(const double* num, const double* den, double* out, cudaStream_t s);
void to_fp32_scaled(long long n, const double* x, const double* scale, bool invert, float* y, cudaStream_t s);
void to_fp64_scaled(long long n, const float* x, const double* scale, double* y, cudaStream_t s);
// x *= dinv (element-wise)
void jacobi_apply(long long n, const double* dinv, double* x, cudaStream_t s);
void reciprocal(long long n, const double* d, double* dinv64, float* dinv32, cudaStream_t s);
// z[i] in [-1, 1) from a hash of (i, seed) (splitmix64 finaliser): a field uncorrelated with
// any residual, for the fault injection of the learned solvers
void fill_noise(long long n, double* z, unsigned long long seed, cudaStream_t s);

}  // namespace nhmf
