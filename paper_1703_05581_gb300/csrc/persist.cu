// Persistence score (Section 5): the normalised series scored 1/0 per sample
// against a cutoff (k_normalise_* writes the bits), folded by the same FFA
// with integer adds (launch_fold, int8 input), and summed per trial over the
// best boxcar window of that trial's record.  The last FFA stage is applied
// while summing, as the scorer does: trial k's profile is head row k>>1 plus
// tail row M/2 + (k>>1) read ceil(k/2) bins further on (cyclic).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace ffa {
namespace {

__global__ void __launch_bounds__(256) k_persist(const int32_t* __restrict__ plane, int64_t m_rows,
                                                 int64_t p0, int64_t ld, const ffa_record* __restrict__ rec,
                                                 uint32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t half = m_rows >> 1;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < m_rows; k += n_warps) {
        const ffa_record r = rec[k];
        const int64_t w = r.width, ph = r.phase;
        const int32_t* h = m_rows > 1 ? plane + (k >> 1) * ld : plane;
        const int32_t* t = m_rows > 1 ? plane + (half + (k >> 1)) * ld : nullptr;
        const int64_t sh = ((k + 1) >> 1) % p0;
        uint32_t acc = 0;
        for (int64_t i = lane; i < w; i += 32) {
            const int64_t j = (ph + i) % p0;
            int32_t v = h[j];
            if (t) {
                int64_t jt = j + sh;
                if (jt >= p0) jt -= p0;
                v += t[jt];
            }
            acc += (uint32_t)v;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[k] = acc;
    }
}

}  // namespace

ffa_status launch_persist(const int32_t* d_bplane, int64_t m_rows, int64_t p0, int64_t ld,
                          const ffa_record* d_rec, uint32_t* d_persist, cudaStream_t st) {
    if (m_rows <= 0) return FFA_OK;
    const int64_t blocks = (m_rows * 32 + 255) / 256;
    const int grid = (int)(blocks < sm_count() * 8 ? blocks : sm_count() * 8);
    k_persist<<<grid, 256, 0, st>>>(d_bplane, m_rows, p0, ld, d_rec, d_persist);
    FFA_LAUNCH_CHECK("k_persist");
    count_launch(1);
    return FFA_OK;
}

}  // namespace ffa
