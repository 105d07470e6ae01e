// teuk_noalloc.cu -- an allocation-free way to reduce waveform records to the
// sin(theta)-weighted scalar w_n.
//
// Who needs it: code that may not allocate device memory at all.  Two common
// cases are a host application that hands all device memory to its own pool at
// start-up (so any later cudaMalloc fails or fragments that pool), and a
// latency-critical loop in which a driver allocation, which can synchronize the
// device, is not acceptable.  teuk_extract allocates a small temporary device
// buffer for the same reduction; this entry point uses a fixed device array
// instead and allocates nothing.
//
// The scratch is one file-scope __device__ array of kNoAllocMaxRecords double2
// values (1 MiB), present on every GPU that loads the library until the process
// exits.  Host code never passes the array's name to a kernel (in host code that
// name is only a stand-in): every call looks up the array's device address on the
// current device with cudaGetSymbolAddress (which allocates nothing), so the address
// is never stale, for example after a device reset.
#include <string>

#include "teuk.h"
#include "teuk_internal.cuh"

namespace teuk {
void set_global_error(const std::string& msg);
}

namespace {

constexpr int64_t kNoAllocMaxRecords = TEUK_NOALLOC_MAX_RECORDS;

static __device__ __align__(256) double2 g_wave_sum_scratch[kNoAllocMaxRecords];

// Device address of the scratch array on the current device.  Under lazy module
// loading the first lookup on a device is what loads the module and places the array.
cudaError_t scratch_address(double2** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_wave_sum_scratch);
    if (e != cudaSuccess) return e;
    *out = (double2*)p;
    return cudaSuccess;
}

}  // namespace

extern "C" teuk_status teuk_waveform_sum_noalloc(const double* wave_dev, int64_t n_records,
                                                 int n_theta, double* out_host,
                                                 void* cuda_stream) {
    if (n_records < 0 || n_records > kNoAllocMaxRecords) {
        teuk::set_global_error("teuk_waveform_sum_noalloc: n_records=" + std::to_string(n_records) +
                               " is outside [0, " + std::to_string(kNoAllocMaxRecords) +
                               "], the size of the fixed scratch array");
        return TEUK_EINVAL;
    }
    if (n_theta < 1 || n_theta > 1024) {
        teuk::set_global_error("teuk_waveform_sum_noalloc: n_theta must be in [1, 1024]");
        return TEUK_EINVAL;
    }
    // the lookup comes first, so that a call with no records places the array on this
    // device: the warm-up to make before a region that must not allocate
    double2* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        teuk::set_global_error(std::string("teuk_waveform_sum_noalloc: ") + cudaGetErrorString(e));
        return TEUK_ECUDA;
    }
    if (n_records == 0) return TEUK_OK;
    if (!wave_dev || !out_host) {
        teuk::set_global_error("teuk_waveform_sum_noalloc: NULL input or output");
        return TEUK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    {
        const double dth = 3.141592653589793238462643 / (double)n_theta;
        // every output element is written, so nothing has to be cleared first
        teuk::launch_wave_sum(st, (const double2*)wave_dev, n_records, n_theta, dth, 0, n_records,
                              scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, scratch, sizeof(double2) * n_records,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        teuk::set_global_error(std::string("teuk_waveform_sum_noalloc: ") + cudaGetErrorString(e));
        return TEUK_ECUDA;
    }
    return TEUK_OK;
}
