// Small kernels of libheom: the FP64 observable record of sigma_0 and the state scatter / gather
// through the host layout.
#include <cuda_runtime.h>

#include <cstdint>

#include "heom_internal.h"

// ------------------------------------------------------------------------------------------------
// small kernels

namespace heom {

__device__ __forceinline__ double2 ld_any(const StateView &s, int E, int Ep, int u_split, int body_fp32, int64_t v,
                                          int64_t e) {
  if (v < u_split) return s.head[v * E + e];
  if (body_fp32) {
    const float2 f = reinterpret_cast<const float2 *>(s.body)[(v - u_split) * Ep + e];
    return make_double2(f.x, f.y);
  }
  return reinterpret_cast<const double2 *>(s.body)[(v - u_split) * Ep + e];
}

// Element e = i n + j of ADO v in the run's layout: matrix tiles, or (vec) column 0 only.
__device__ __forceinline__ double2 ld_elem(const StateView &s, int n, int Ep, int u_split, int body_fp32, int vec,
                                           int64_t v, int64_t e) {
  if (!vec) return ld_any(s, n * n, Ep, u_split, body_fp32, v, e);
  const int64_t i = e / n, j = e - i * n;
  if (j != 0) return make_double2(0.0, 0.0);
  return ld_any(s, n, n, u_split, body_fp32, v, i);
}

// One observable record of sigma_0 (FP64): populations, trace, dipole correlation, Hermiticity.
__global__ void record_kernel(StateView y, int u_split, int body_fp32, int vec, int n, const double *w, double *records,
                              int64_t *rec_count, int64_t max_records) {
  // one warp: lane a handles rows a, a + 32, ...; sums and the maximum are reduced across the warp
  const int lane = threadIdx.x & 31;
  const int64_t idx = *rec_count;
  if (idx >= max_records) return;
  const int E = n * n;
  double *rec = records + idx * (n + 5);
  double tr = 0, ti = 0, cr = 0, ci = 0, herm = 0;
  for (int a = lane; a < n; a += 32) {
    const double2 d = ld_elem(y, n, E, u_split, body_fp32, vec, 0, (int64_t)a * n + a);
    rec[a] = d.x;
    tr += d.x;
    ti += d.y;
    const double2 c0 = ld_elem(y, n, E, u_split, body_fp32, vec, 0, (int64_t)a * n);
    cr += w[a] * c0.x;
    ci += w[a] * c0.y;
    for (int b = 0; b < n; ++b) {
      const double2 x = ld_elem(y, n, E, u_split, body_fp32, vec, 0, (int64_t)a * n + b);
      const double2 z = ld_elem(y, n, E, u_split, body_fp32, vec, 0, (int64_t)b * n + a);
      herm = fmax(herm, hypot(x.x - z.x, x.y + z.y));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_down_sync(0xffffffffu, tr, o);
    ti += __shfl_down_sync(0xffffffffu, ti, o);
    cr += __shfl_down_sync(0xffffffffu, cr, o);
    ci += __shfl_down_sync(0xffffffffu, ci, o);
    herm = fmax(herm, __shfl_down_sync(0xffffffffu, herm, o));
  }
  if (lane == 0) {
    rec[n] = tr;
    rec[n + 1] = ti;
    rec[n + 2] = cr;
    rec[n + 3] = ci;
    rec[n + 4] = herm;
    *rec_count = idx + 1;
  }
}

__global__ void scatter_kernel(StateView dst, int Ep, int u_split, int body_fp32, int vec, int n, int64_t u0, int64_t count,
                               const double *re, const double *im) {
  const int64_t E = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count * E; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / E;
    int64_t e = t - c * E;
    const int64_t v = u0 + c;
    int64_t TE = E, TP = Ep;
    if (vec) {  // column 0 only (the host checked that the rest is zero)
      if (e % n != 0) continue;
      e /= n;
      TE = n;
      TP = n;
    }
    if (v < u_split) {
      dst.head[v * TE + e] = make_double2(re[t], im[t]);
    } else if (body_fp32) {
      reinterpret_cast<float2 *>(dst.body)[(v - u_split) * TP + e] = make_float2((float)re[t], (float)im[t]);
    } else {
      reinterpret_cast<double2 *>(dst.body)[(v - u_split) * TP + e] = make_double2(re[t], im[t]);
    }
  }
}

__global__ void gather_kernel(StateView src, int Ep, int u_split, int body_fp32, int vec, int n, int64_t u0, int64_t count,
                              double *re, double *im) {
  const int64_t E = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count * E; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / E, e = t - c * E;
    const double2 d = ld_elem(src, n, Ep, u_split, body_fp32, vec, u0 + c, e);
    re[t] = d.x;
    im[t] = d.y;
  }
}

}  // namespace heom
