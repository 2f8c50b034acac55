// Distances between LDP descriptors (region / window histograms used as
// feature vectors): every query row q_a against every gallery row g_b,
//   L1            sum_d |q - g|                    (exact, uint64 out)
//   intersection  sum_d min(q, g)                  (exact, uint64 out)
//   chi-square    sum_{q+g>0} (q - g)^2 / (q + g)  (fp32 out)
// A CTA owns a 64 x 64 block of (query, gallery) pairs; 256 threads hold
// 4 x 4 pairs each (queries ty + 16 i, gallery rows tx + 16 j).  The
// descriptors pass through shared memory in chunks of 32 components, rows
// padded to 33 words: the 16 gallery rows a warp reads sit in 16 different
// banks, the two query rows are broadcasts.  Integer metrics sum a chunk in
// 32 bits (exact for counts below 2^27) and widen to 64 bits per chunk,
// two components per add; L1 is computed as sum q + sum g - 2 sum min(q, g)
// (|a - b| = a + b - 2 min(a, b)), the row sums gathered from the same
// shared-memory chunks.  Chi-square converts counts to fp32 (exact below
// 2^24) and uses the hardware reciprocal of max(q + g, 1), so an empty bin
// adds exactly 0.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ldp_launch.h"

namespace ldp {

namespace {

constexpr int kTile = 64, kChunk = 32;

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int METRIC>
__global__ void __launch_bounds__(256) k_distance(const uint32_t* __restrict__ Q, int nq, int ldq,
                                                  const uint32_t* __restrict__ G, int ng, int ldg, int D,
                                                  void* out, int ldo) {
    using T = std::conditional_t<METRIC == LDP_DIST_CHI2, float, uint32_t>;
    __shared__ T qs[kTile][kChunk + 1], gs[kTile][kChunk + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int a0 = blockIdx.y * kTile, b0 = blockIdx.x * kTile;
    __shared__ uint64_t rsum[2][kTile];  // L1: row sums of the CTA's query and gallery rows
    uint64_t acc[4][4] = {};
    float facc[4][4] = {};
    uint64_t my_sum = 0;  // L1: threads 0..127 sum one query (0..63) or gallery (64..127) row
    for (int k0 = 0; k0 < D; k0 += kChunk) {
        for (int e = threadIdx.x; e < kTile * kChunk; e += blockDim.x) {
            const int r = e / kChunk, d = e % kChunk, k = k0 + d;
            const uint32_t qv = (a0 + r < nq && k < D) ? __ldg(Q + (size_t)(a0 + r) * ldq + k) : 0u;
            const uint32_t gv = (b0 + r < ng && k < D) ? __ldg(G + (size_t)(b0 + r) * ldg + k) : 0u;
            qs[r][d] = (T)qv;
            gs[r][d] = (T)gv;
        }
        __syncthreads();
        if constexpr (METRIC == LDP_DIST_L1) {
            if (threadIdx.x < 2 * kTile) {
                const uint32_t* row = threadIdx.x < kTile ? &qs[threadIdx.x][0] : &gs[threadIdx.x - kTile][0];
                uint32_t s = 0;
#pragma unroll
                for (int d = 0; d < kChunk; ++d) s += row[d];
                my_sum += s;
            }
        }
        uint32_t part[4][4] = {};
#pragma unroll 4
        for (int d = 0; d < kChunk; d += 2) {
            T qv[2][4], gv[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int i = 0; i < 4; ++i) qv[h][i] = qs[ty + 16 * i][d + h];
#pragma unroll
                for (int j = 0; j < 4; ++j) gv[h][j] = gs[tx + 16 * j][d + h];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if constexpr (METRIC == LDP_DIST_CHI2) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float t = qv[h][i] - gv[h][j], s = qv[h][i] + gv[h][j];
                            facc[i][j] = fmaf(t * t, rcp_approx(fmaxf(s, 1.0f)), facc[i][j]);
                        }
                    } else {
                        part[i][j] += min(qv[0][i], gv[0][j]) + min(qv[1][i], gv[1][j]);
                    }
                }
        }
        if constexpr (METRIC != LDP_DIST_CHI2) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
        }
        __syncthreads();
    }
    if constexpr (METRIC == LDP_DIST_L1) {
        if (threadIdx.x < 2 * kTile) rsum[threadIdx.x / kTile][threadIdx.x % kTile] = my_sum;
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int a = a0 + ty + 16 * i;
        if (a >= nq) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + tx + 16 * j;
            if (b >= ng) continue;
            if constexpr (METRIC == LDP_DIST_CHI2)
                static_cast<float*>(out)[(size_t)a * ldo + b] = facc[i][j];
            else if constexpr (METRIC == LDP_DIST_L1)
                static_cast<uint64_t*>(out)[(size_t)a * ldo + b] =
                    rsum[0][ty + 16 * i] + rsum[1][tx + 16 * j] - 2 * acc[i][j];
            else
                static_cast<uint64_t*>(out)[(size_t)a * ldo + b] = acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_distance(const uint32_t* q, int nq, int ldq, const uint32_t* g, int ng, int ldg, int D,
                            int metric, void* out, int ldo, cudaStream_t s) {
    dim3 grid((ng + kTile - 1) / kTile, (nq + kTile - 1) / kTile);
    switch (metric) {
        case LDP_DIST_L1: k_distance<LDP_DIST_L1><<<grid, 256, 0, s>>>(q, nq, ldq, g, ng, ldg, D, out, ldo); break;
        case LDP_DIST_INTERSECT:
            k_distance<LDP_DIST_INTERSECT><<<grid, 256, 0, s>>>(q, nq, ldq, g, ng, ldg, D, out, ldo);
            break;
        case LDP_DIST_CHI2: k_distance<LDP_DIST_CHI2><<<grid, 256, 0, s>>>(q, nq, ldq, g, ng, ldg, D, out, ldo); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ldp

// C-ABI entry point (include/ldp.h).
extern "C" {

int ldp_hist_distance(const uint32_t* d_q, int nq, int ldq, const uint32_t* d_g, int ng, int ldg, int D,
                      int metric, void* d_out, int ldo, void* stream) {
    if (!d_q || !d_g || !d_out) return ldp::report_error(LDP_EINVAL, "descriptor or output pointer is NULL");
    if (nq < 1 || ng < 1 || D < 1) return ldp::report_error(LDP_EINVAL, "nq, ng and D must be at least 1");
    if (nq > (1 << 22) || ng > (1 << 30)) return ldp::report_error(LDP_EINVAL, "nq or ng too large");
    if (ldq < D || ldg < D || ldo < ng) return ldp::report_error(LDP_EINVAL, "leading dimension too small");
    if (metric < LDP_DIST_L1 || metric > LDP_DIST_CHI2) return ldp::report_error(LDP_EINVAL, "metric must be one of LDP_DIST_*");
    ldp::Range range("ldp.hist_distance");
    cudaError_t e = ldp::launch_distance(d_q, nq, ldq, d_g, ng, ldg, D, metric, d_out, ldo,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ldp::report_cuda(e, "distance kernel");
    return LDP_OK;
}

}  // extern "C"
