// U-Net preconditioner state (see unet.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace nhmf {

struct UNetLayer {
  int kind;                  // 0 conv, 1 down (stride 2), 2 up (transposed stride 2)
  int cin, cout;
  long long woff, boff;      // offsets in the flat parameter array
  __nv_bfloat16* wf;         // forward weights [27][16][16] (tap, co, ci)
  __nv_bfloat16* wb;         // backward-data weights [27][16][16]
};

struct UNet {
  int M0 = 0, M1 = 0, M2 = 0;
  long long N0 = 0, N1 = 0, N2 = 0;
  long long nparams = 0;
  int step = 0;
  UNetLayer L[11];
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  __nv_bfloat16 *x16 = nullptr, *a0 = nullptr, *s0 = nullptr, *d1 = nullptr, *s1 = nullptr, *d2 = nullptr,
                *m2 = nullptr, *u1 = nullptr, *t1 = nullptr, *u0 = nullptr, *t0 = nullptr;
  __nv_bfloat16 *g0a = nullptr, *g0b = nullptr, *g0c = nullptr, *g1a = nullptr, *g1b = nullptr, *g1c = nullptr,
                *g2a = nullptr, *g2b = nullptr;
  float* y = nullptr;          // [3][N0] network output
  float* partial = nullptr;    // weight-gradient partials
  double* sc = nullptr;        // device scalars
  float* pairs = nullptr;      // [cap][2][3][N0]: normalised input, normalised target
  int cap = 0, npairs = 0;
  unsigned* status = nullptr;  // the context's device status word
};

}  // namespace nhmf
