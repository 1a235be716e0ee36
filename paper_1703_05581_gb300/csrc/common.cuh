// Shared device/host helpers of the FFA library (no method arithmetic here
// beyond order-preserving key transforms and error plumbing).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ffa.h"

namespace ffa {

// Thread-local error message, set together with a failing ffa_status.
void set_error(const std::string& msg);
ffa_status fail(ffa_status s, const std::string& msg);
ffa_status cuda_fail(cudaError_t e, const char* where);

#define FFA_CUDA_TRY(call)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::ffa::cuda_fail(e_, #call); \
    } while (0)

#define FFA_LAUNCH_CHECK(what)                                      \
    do {                                                            \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return ::ffa::cuda_fail(e_, what);   \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Order-preserving unsigned keys: a < b  <=>  key(a) < key(b) (no NaNs).
__device__ __forceinline__ uint32_t fkey(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}
__device__ __forceinline__ uint64_t dkey(double d) {
    uint64_t u = (uint64_t)__double_as_longlong(d);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(uint64_t k) {
    uint64_t u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}
__host__ __device__ __forceinline__ uint32_t ikey(int32_t v) { return (uint32_t)v ^ 0x80000000u; }

// Record a device-side check failure without trapping.
__device__ __forceinline__ void dev_fail(int32_t* d_status, int32_t code) {
    if (d_status) atomicCAS(d_status, 0, code);
}

}  // namespace ffa
