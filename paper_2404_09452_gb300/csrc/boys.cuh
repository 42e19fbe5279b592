// Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt in FP64 on the device.
//
// T < BOYS_TMAX: F_M at the nearest grid point T_k = k h (h = 0.1, |d| <= h/2)
// from the Taylor series F_M(T_k + d) = sum_j F_{M+j}(T_k) (-d)^j / j!
// (dF_m/dT = -F_{m+1}), nine terms, so the truncation is below
// (h/2)^9 / 9! ~ 5e-18 relative; e^-T from the same expansion of e^-T_k; then
// the downward recursion F_m = (2T F_{m+1} + e^-T) / (2m+1), which is stable.
// T >= BOYS_TMAX: F_0 = sqrt(pi/T)/2 (erf(sqrt(T)) = 1 to double precision
// beyond T = 40) and the upward recursion F_{m+1} = ((2m+1) F_m - e^-T)/(2T),
// stable for T > m.
// The grid values are generated on the host by `boys_table_host` (series in
// long double) and live in device global memory.
#pragma once

#include <cuda_runtime.h>

namespace dfjk {

constexpr int BOYS_MMAX = 8;     // highest order any kernel asks for
constexpr int BOYS_TAYLOR = 9;   // Taylor terms
constexpr int BOYS_NCOL = BOYS_MMAX + BOYS_TAYLOR + 1;  // orders 0..16, then e^-T_k
constexpr int BOYS_NPT = 401;    // T_k = 0, 0.1, ..., 40
constexpr double BOYS_H = 0.1;
constexpr double BOYS_TMAX = 40.0;

// Host: fills tab[BOYS_NPT][BOYS_NCOL + 1]; column BOYS_NCOL holds e^-T_k.
void boys_table_host(double *tab);
// Device copy of the table for the current device (built on first use).
const double *boys_table_device();
// The same table rounded to FP32, for the FP32 integral path.
const float *boys_table_device_f32();

// FP32 Boys function for the single-precision integrals of small shell pairs:
// the same grid and expansion with five Taylor terms ((h/2)^5/5! ~ 3e-9, below
// FP32 rounding), the FP32 table, and the same downward / upward recursions.
template <int M>
__device__ __forceinline__ void boys_eval(float T, const float *__restrict__ tab, float *F) {
  constexpr int NT = 5;
  if (T < (float)BOYS_TMAX) {
    const int k = __float2int_rn(T * (float)(1.0 / BOYS_H));
    const float x = (float)k * (float)BOYS_H - T;
    const float *row = tab + k * (BOYS_NCOL + 1);
    float f = __ldg(row + M + NT - 1);
    float e = 1.0f;
#pragma unroll
    for (int j = NT - 2; j >= 0; --j) {
      const float xj = x * (1.0f / (j + 1));
      f = fmaf(f, xj, __ldg(row + M + j));
      e = fmaf(e, xj, 1.0f);
    }
    e *= __ldg(row + BOYS_NCOL);
    F[M] = f;
    const float t2 = T + T;
#pragma unroll
    for (int m = M - 1; m >= 0; --m) F[m] = fmaf(t2, F[m + 1], e) * (1.0f / (2 * m + 1));
  } else {
    const float e = expf(-T);
    const float r = 1.0f / (T + T);
    F[0] = 0.88622692545275801365f * rsqrtf(T);
#pragma unroll
    for (int m = 0; m < M; ++m) F[m + 1] = fmaf((float)(2 * m + 1), F[m], -e) * r;
  }
}

template <int M>
__device__ __forceinline__ void boys_eval(double T, const double *__restrict__ tab, double *F) {
  if (T < BOYS_TMAX) {
    const int k = __double2int_rn(T * (1.0 / BOYS_H));
    const double x = (double)k * BOYS_H - T;  // = -d
    const double *row = tab + k * (BOYS_NCOL + 1);
    // Horner for both sums with the shared factors x/(j+1).
    double f = __ldg(row + M + BOYS_TAYLOR - 1);
    double e = 1.0;
#pragma unroll
    for (int j = BOYS_TAYLOR - 2; j >= 0; --j) {
      const double xj = x * (1.0 / (j + 1));
      f = fma(f, xj, __ldg(row + M + j));
      e = fma(e, xj, 1.0);
    }
    e *= __ldg(row + BOYS_NCOL);
    F[M] = f;
    const double t2 = T + T;
#pragma unroll
    for (int m = M - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], e) * (1.0 / (2 * m + 1));
  } else {
    const double e = exp(-T);
    const double r = 1.0 / (T + T);
    F[0] = 0.88622692545275801365 * rsqrt(T);  // sqrt(pi)/2
#pragma unroll
    for (int m = 0; m < M; ++m) F[m + 1] = fma((double)(2 * m + 1), F[m], -e) * r;
  }
}

}  // namespace dfjk
