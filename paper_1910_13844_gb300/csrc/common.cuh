// Shared device/host definitions of the LS library (complex helpers, slot state, errors).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "ls.h"

namespace lsgpu {

// ---------------------------------------------------------------- complex64

__host__ __device__ __forceinline__ float2 c2(float x, float y) { return make_float2(x, y); }
// Complex add/subtract.  On sm_100 and later the two components go through one packed
// add.f32x2 / sub.f32x2 (IEEE round-to-nearest per component, as the scalar adds), which halves
// the issue slots of the FFT butterflies.
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  float2 r;
  asm("{\n .reg .b64 pa, pb, pr;\n mov.b64 pa, {%2, %3};\n mov.b64 pb, {%4, %5};\n"
      " add.rn.f32x2 pr, pa, pb;\n mov.b64 {%0, %1}, pr;\n}\n"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  float2 r;
  asm("{\n .reg .b64 pa, pb, pr;\n mov.b64 pa, {%2, %3};\n mov.b64 pb, {%4, %5};\n"
      " sub.rn.f32x2 pr, pa, pb;\n mov.b64 {%0, %1}, pr;\n}\n"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// conj(a) * b  (the inner-product term <a, b> = sum conj(a) b)
__host__ __device__ __forceinline__ float2 cdotterm(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------- complex128 (plan time only)

__host__ __device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// ---------------------------------------------------------------- solver slots
//
// Every batched kernel works on "slots": one slot is one view of one request
// with its own Krylov vectors.  A kernel runs for slot s only if
// (slots[s].flags & mask) != 0; mask == 0 means "every slot".

enum SlotFlag : unsigned {
  SLOT_ITER = 1u,     // BiCGStab iterating
  SLOT_RESID = 2u,    // needs a true-residual evaluation (start or exit check)
  SLOT_FAR = 4u,      // far field to evaluate
  SLOT_AUX = 8u,      // generic selection used by one-off operations
};

struct SlotDev {
  const float* f;      // potential of this slot's request (N floats)
  unsigned flags;
  int adjoint;         // 1: operator x - G^H (f x)
  int first;           // 1: next p-update starts the recurrence (p = r)
  int iters;
  int status;          // LS_OK / LS_NOT_CONVERGED / LS_BREAKDOWN while running
  int restarts;
  int matvecs;
  int max_iter;
  int checks;          // true-residual evaluations so far (0: the initial one)
  int max_restarts;
  double tol;
  double2 rho, alpha, omega, beta;   // BiCGStab scalars (complex, float64)
  float2 alpha_f, omega_f, beta_f;   // the same rounded to float once per scalar step, for the vector kernels
                                     // (a float64 -> float32 conversion in every thread costs GB300's slow
                                     // float64 pipe)
  double bnorm2, rnorm2, true_rnorm2;
  double rhnorm2;      // ||rh||^2 of the shadow residual (fixed from the last (re)start)
};

// ---------------------------------------------------------------- error handling (host)

void set_last_error(const char* fmt, ...);

}  // namespace lsgpu

#define LS_CUDA_TRY(expr)                                                                 \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess) {                                                              \
      ::lsgpu::set_last_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),     \
                              __FILE__, __LINE__);                                        \
      return (_e == cudaErrorMemoryAllocation) ? LS_ENOMEM : LS_ECUDA;                    \
    }                                                                                     \
  } while (0)
