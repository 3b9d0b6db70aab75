// resample.cu -- linear time resampling of receiver traces between two
// operators with different time steps (the non-inverse-crime study of
// Sec. 6.2: data simulated on a fine grid, reconstructed on a coarse one).
//
// out[k][l] = in(s_k)[l], s_k = s0 + k * ratio (in input samples), linear
// between the two neighbouring input samples and zero outside [0, m_in - 1].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "pact.h"

void pact_note_error(const std::string& msg);

namespace {

__global__ void k_resample(const float* __restrict__ in, int m_in, float* __restrict__ out, int m_out, int L,
                           double s0, double ratio) {
    const size_t n = (size_t)m_out * L;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / L), l = (int)(i % L);
        const double s = s0 + k * ratio;
        float v = 0.f;
        if (s >= 0.0 && s <= (double)(m_in - 1)) {
            const int j = std::min((int)floor(s), m_in - 2 < 0 ? 0 : m_in - 2);
            const double f = s - j;
            const float a = in[(size_t)j * L + l];
            const float b = j + 1 < m_in ? in[(size_t)(j + 1) * L + l] : a;
            v = (float)((1.0 - f) * a + f * b);
        }
        out[i] = v;
    }
}

}  // namespace

extern "C" int pact_resample_traces(const float* in, int m_in, float* out, int m_out, int L, double s0,
                                    double ratio, void* stream) {
    if (!in || !out || m_in < 1 || m_out < 1 || L < 1 || !(ratio > 0.0) || !std::isfinite(s0)) {
        pact_note_error("pact_resample_traces: NULL pointer, empty traces or ratio <= 0");
        return PACT_EINVAL;
    }
    const size_t n = (size_t)m_out * L;
    const unsigned g = (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 8));
    k_resample<<<g, 256, 0, (cudaStream_t)stream>>>(in, m_in, out, m_out, L, s0, ratio);
    if (cudaGetLastError() != cudaSuccess) {
        pact_note_error("pact_resample_traces: launch failed");
        return PACT_ECUDA;
    }
    return PACT_OK;
}
