// heom_propagate_static: a propagation entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: plug-ins and embedded callers whose host application owns
// every device allocation and hands the library no buffer, and latency-critical paths where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.  For them the whole
// device workspace of one small propagation -- link tables, decay sums, the state and the two
// intermediate RK4 copies the stage kernel works in, and the observable records -- lives in one
// file-scope device array owned by the library, of kStaticBytes bytes.  Every GPU that loads the
// library holds that array until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/heom.h"
#include "heom_internal.h"
#include "heom_run.h"

namespace heom {

constexpr size_t kStaticBytes = 32u << 20;  // 32 MiB per device

// The shared scratch array.  Host code must not use its name as an address: the name only stands
// for the device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;  // guards the per-device address table
std::mutex g_call_mu;    // one call at a time in this process: all calls share the array
void *g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_ws on the current device, looked up once per device.
int static_workspace(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("heom_propagate_static: cudaGetDevice: ") + cudaGetErrorString(e));
    return HEOM_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("heom_propagate_static: device ordinal above 63");
    return HEOM_E_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p) {
      set_error(std::string("heom_propagate_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return HEOM_E_CUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return HEOM_OK;
}
}  // namespace

}  // namespace heom

using namespace heom;

extern "C" int heom_propagate_static(const heom_system *sys, const heom_hier *h, int precision,
                                     const double *sigma0_re, const double *sigma0_im, const double *dip_w,
                                     double dt_fs, int64_t n_steps, int64_t obs_stride, void *cuda_stream,
                                     double *records_out, int64_t cap_records, int64_t *written,
                                     double *sigma0_out_re, double *sigma0_out_im) {
  if (!records_out || cap_records < 1 || n_steps < 0 || obs_stride < 0) {
    set_error("heom_propagate_static: need records_out, cap_records >= 1, n_steps >= 0, obs_stride >= 0");
    return HEOM_E_ARG;
  }
  const int64_t max_records = 1 + (obs_stride > 0 ? n_steps / obs_stride : 0);
  if (max_records > cap_records) {
    set_error("heom_propagate_static: cap_records below 1 + n_steps / obs_stride");
    return HEOM_E_ARG;
  }
  size_t need = 0;
  int rc = heom_run_bytes(sys, h, precision, max_records, &need);
  if (rc != HEOM_OK) return rc;
  if (need > kStaticBytes) {
    set_error("heom_propagate_static: the run needs " + std::to_string(need) + " bytes of device workspace, above "
              "the static limit of " + std::to_string(kStaticBytes) + " bytes (32 MiB); use heom_run_create");
    return HEOM_E_NOMEM;
  }
  void *ws = nullptr;
  rc = static_workspace(&ws);
  if (rc != HEOM_OK) return rc;
  std::lock_guard<std::mutex> call_lock(g_call_mu);
  // heom_run_create zeroes the state copies and the record counter it uses in the array, so what
  // an earlier call left there does not leak into this one.
  heom_run *r = nullptr;
  ++g_tune_suppress;  // no autotuning here: cached schedules or the default
  rc = heom_run_create(sys, h, precision, max_records, sigma0_re, sigma0_im, dip_w, ws, kStaticBytes, cuda_stream,
                       &r);
  --g_tune_suppress;
  if (rc != HEOM_OK) {
    // creation may have queued uploads into the array before it failed: let them finish before the
    // lock is released, so that the next call does not reuse the array under them
    cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(cuda_stream));
    return rc;
  }
  rc = heom_propagate(r, dt_fs, n_steps, obs_stride);
  if (rc == HEOM_OK) rc = heom_observables(r, records_out, cap_records, written);
  if (rc == HEOM_OK && sigma0_out_re && sigma0_out_im) rc = heom_get_sigma0(r, sigma0_out_re, sigma0_out_im);
  if (rc != HEOM_OK) {
    // on an error, stages may still be queued on the caller's stream and on the run's side stream
    // (the FP64 head launches of a mixed run): wait for both before the array is released; the
    // message of the first failure is kept
    const std::string msg = heom_last_error();
    if (r->side) cudaStreamSynchronize(r->side);
    cudaStreamSynchronize(r->stream);
    set_error(msg);
  }
  heom_run_destroy(r);
  return rc;
}
