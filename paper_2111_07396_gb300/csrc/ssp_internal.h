// ssp_internal.h -- what the C ABI translation unit (ssp_api.cu) offers the
// library's other host code (the serving loop in ssp_server.cu).
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/ssp.h"

namespace ssp_internal {

// sets the calling thread's last error and returns code
int fail(int code, const char *msg);
std::string last_error();
void clear_error();

int check_params(const ssp_params &p);
// one object's host arrays: 4 <= n <= 65535 and the value rules of
// ssp_periodogram
int check_one_object(const ssp_params &p, const double *t, const double *y, const double *dy,
                     int64_t n);
int check_freq(const double *freq_grid, int64_t n_freq);

// the device pipeline of ssp_periodogram_device (device t, y, dy, freq and
// outputs; host n_per_object), enqueued on s
// SSP_TESTING=1 in the environment: tuning overrides and fault injection on
bool testing();
// device allocation of the library's workspaces: cudaMallocAsync, or an
// injected out-of-memory failure (ssp_test_fault, SSP_FAULT_ALLOC)
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s);
// serving: true when the next batch is to be treated as stalled
// (ssp_test_fault, SSP_FAULT_STALL)
bool stall_injected();
// serving: true when the next upload of a request is to fail
// (ssp_test_fault, SSP_FAULT_UPLOAD)
bool upload_fault_injected();

// device bytes that run() takes from the stream-ordered pool for this batch
// (workspace, slabs), or a negative status
int64_t device_bytes(const int64_t *n_per_object, int64_t n_objects, int64_t n_freq,
                     ssp_variant variant, const ssp_params &p);

int run(const double *t, const double *y, const double *dy, const int64_t *n_per_object,
        int64_t n_objects, const double *freq, int64_t n_freq, ssp_variant variant,
        const ssp_params &p, void *out_power, double *out_best, cudaStream_t s);

}  // namespace ssp_internal
