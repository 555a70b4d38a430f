// Sherman-Morrison update of the inverse Slater matrices of a batch of
// walkers after one accepted move each (Sec. VI.D: the O(N^2) update the
// paper measures as the second bottleneck of the step).
//
// Row j of D (D[j][l] = psi_l(r_j)) is replaced by the new orbital row psi'.
// With Dinv[l][k] = (D^{-1})_{lk} and w_k = sum_l psi'_l Dinv[l][k]
// (w_j = xi, the acceptance ratio),
//     Dinv'[l][k] = Dinv[l][k] - Dinv[l][j] (w_k - delta_jk) / w_j.
// Two HBM-bound passes per walker: a GEMV for w (reads Dinv once; also keeps
// column j aside) and the rank-1 update (reads and writes Dinv once), i.e.
// 12 n^2 bytes per walker update in FP32.
#include <cuda_runtime.h>

#include "blip_internal.h"

namespace blip {

namespace {

constexpr int SM_THREADS = 256;
constexpr int SM_ROWS = 8;      // rows of Dinv per thread in the rank-1 pass

// w[wk][k] = sum_l rows[wk][l] Dinv[wk][l][k]; colj[wk][l] = Dinv[wk][l][j].
__global__ void __launch_bounds__(SM_THREADS) sm_gemv_kernel(int n, const float *__restrict__ dinv,
                                                             const float *__restrict__ rows,
                                                             const int *__restrict__ cols,
                                                             float *__restrict__ work)
{
    __shared__ float srow[SM_THREADS];
    const int wk = blockIdx.y;
    const int j = cols[wk];
    if (j < 0 || j >= n) return;                       // no accepted move for this walker
    const float *D = dinv + (size_t)wk * n * n;
    const float *r = rows + (size_t)wk * n;
    float *w = work + (size_t)wk * 2 * n;
    const int k = blockIdx.x * SM_THREADS + threadIdx.x;
    float acc = 0.0f;
    for (int l0 = 0; l0 < n; l0 += SM_THREADS) {
        const int m = min(SM_THREADS, n - l0);
        __syncthreads();
        if (threadIdx.x < m) srow[threadIdx.x] = r[l0 + threadIdx.x];
        __syncthreads();
        if (k < n) {
            const float *Dl = D + (size_t)l0 * n + k;
#pragma unroll 8
            for (int i = 0; i < m; ++i) acc = fmaf(srow[i], Dl[(size_t)i * n], acc);
        }
    }
    if (k < n) {
        w[k] = acc;
        w[n + k] = D[(size_t)k * n + j];                  // column j, kept before the update
    }
}

// Dinv[l][k] -= colj[l] (w_k - delta_jk) / w_j.
__global__ void __launch_bounds__(SM_THREADS) sm_rank1_kernel(int n, float *__restrict__ dinv,
                                                              const int *__restrict__ cols,
                                                              const float *__restrict__ work)
{
    const int wk = blockIdx.z;
    const int j = cols[wk];
    if (j < 0 || j >= n) return;
    const int k = blockIdx.x * SM_THREADS + threadIdx.x;
    if (k >= n) return;
    const float *w = work + (size_t)wk * 2 * n;
    const float inv_xi = 1.0f / w[j];
    const float f = (w[k] - (k == j ? 1.0f : 0.0f)) * inv_xi;
    float *D = dinv + (size_t)wk * n * n;
    const int l0 = blockIdx.y * SM_ROWS;
#pragma unroll
    for (int i = 0; i < SM_ROWS; ++i) {
        const int l = l0 + i;
        if (l < n) D[(size_t)l * n + k] = fmaf(-w[n + l], f, D[(size_t)l * n + k]);
    }
}

}  // namespace

cudaError_t launch_sm_update(int n_walkers, int n, float *dinv, const float *rows, const int *cols,
                             float *work, cudaStream_t stream)
{
    const dim3 g1((n + SM_THREADS - 1) / SM_THREADS, n_walkers);
    sm_gemv_kernel<<<g1, SM_THREADS, 0, stream>>>(n, dinv, rows, cols, work);
    const dim3 g2((n + SM_THREADS - 1) / SM_THREADS, (n + SM_ROWS - 1) / SM_ROWS, n_walkers);
    sm_rank1_kernel<<<g2, SM_THREADS, 0, stream>>>(n, dinv, cols, work);
    return cudaGetLastError();
}

}  // namespace blip
