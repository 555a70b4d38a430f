// Sherman-Morrison update of the inverse Slater matrices of a batch of
// walkers after one accepted move each (Sec. VI.D: the O(N^2) update the
// paper measures as the second bottleneck of the step).
//
// Row j of D (D[j][l] = psi_l(r_j)) is replaced by the new orbital row psi'.
// With Dinv[l][k] = (D^{-1})_{lk} and w_k = sum_l psi'_l Dinv[l][k]
// (w_j = xi, the acceptance ratio),
//     Dinv'[l][k] = Dinv[l][k] - Dinv[l][j] (w_k - delta_jk) / w_j.
// For n <= 1024 (the TiO2 cell's 768 electrons of one spin) the update is
// one read and one write of Dinv, 8 n^2 bytes per walker in FP32:
//   1. sm_column_kernel, one warp per walker: column j of Dinv and
//      w_j = sum_l psi'_l Dinv[l][j] (the ratio), kept aside;
//   2. sm_fused_kernel, one block per (walker, 32 columns): 16 warps hold
//      the block's n x 32 slice of Dinv in registers (ceil(n / 16) rows each,
//      a lane per column; two blocks fit an SM, so one block's loads overlap
//      the other's stores), form w_k for their columns (partial sums over the
//      warps added in a fixed order), then update the slice in registers and
//      write it back.
// Larger n takes two passes: a GEMV for w (reads Dinv once; also keeps
// column j aside) and the rank-1 update (reads and writes Dinv once), 12 n^2
// bytes per walker.
#include <cuda_runtime.h>

#include "blip_internal.h"

namespace blip {

namespace {

constexpr int SM_THREADS = 256;
constexpr int SM_ROWS = 8;      // rows of Dinv per thread in the rank-1 pass

// w[wk][k] = sum_l rows[wk][l] Dinv[wk][l][k]; colj[wk][l] = Dinv[wk][l][j].
// A block covers 32 columns (one coalesced 128-byte segment per row) and
// splits the rows over SM_PARTS warps; the partial sums meet in shared
// memory in a fixed order.
constexpr int SM_PARTS = 8;

__global__ void __launch_bounds__(32 * SM_PARTS) sm_gemv_kernel(int n, const float *__restrict__ dinv,
                                                                const float *__restrict__ rows,
                                                                const int *__restrict__ cols,
                                                                float *__restrict__ work)
{
    __shared__ float part[SM_PARTS][32];
    const int wk = blockIdx.y;
    const int j = cols[wk];
    if (j < 0 || j >= n) return;                       // no accepted move for this walker
    const float *D = dinv + (size_t)wk * n * n;
    const float *r = rows + (size_t)wk * n;
    float *w = work + (size_t)wk * 2 * n;
    const int lane = threadIdx.x & 31, pw = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    float acc = 0.0f;
    if (k < n) {
        const int l0 = (int)((long long)n * pw / SM_PARTS), l1 = (int)((long long)n * (pw + 1) / SM_PARTS);
#pragma unroll 8
        for (int l = l0; l < l1; ++l) acc = fmaf(__ldg(r + l), D[(size_t)l * n + k], acc);
    }
    part[pw][lane] = acc;
    __syncthreads();
    if (pw == 0 && k < n) {
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < SM_PARTS; ++q) s += part[q][lane];
        w[k] = s;
    }
    // column j, kept before the update: rows k of this block's range, by warp 1
    if (pw == 1 && k < n) w[n + k] = D[(size_t)k * n + j];
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

constexpr int FU_WARPS = 16;                 // warps per fused block
constexpr int FU_MAX_ROWS = 64;              // rows per warp: n <= 1024

// work[wk][n + l] = Dinv[l][j]; work[wk][j] = w_j = sum_l psi'_l Dinv[l][j].
__global__ void __launch_bounds__(32) sm_column_kernel(int n, const float *__restrict__ dinv,
                                                       const float *__restrict__ rows,
                                                       const int *__restrict__ cols,
                                                       float *__restrict__ work)
{
    const int wk = blockIdx.x;
    const int j = cols[wk];
    if (j < 0 || j >= n) return;
    const float *D = dinv + (size_t)wk * n * n;
    const float *r = rows + (size_t)wk * n;
    float *w = work + (size_t)wk * 2 * n;
    const int lane = threadIdx.x;
    float acc = 0.0f;
    for (int l = lane; l < n; l += 32) {
        const float d = D[(size_t)l * n + j];
        w[n + l] = d;
        acc = fmaf(__ldg(r + l), d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) w[j] = acc;
}

// One block per (walker, 32 columns): the slice stays in registers between
// the product w_k = sum_l psi'_l Dinv[l][k] and the update
// Dinv[l][k] -= Dinv[l][j] (w_k - delta_jk) / w_j.
template <int RPW>
__global__ void __launch_bounds__(32 * FU_WARPS, 2) sm_fused_kernel(int n, float *__restrict__ dinv,
                                                                 const float *__restrict__ rows,
                                                                 const int *__restrict__ cols,
                                                                 const float *__restrict__ work)
{
    __shared__ float part[FU_WARPS][32];
    const int wk = blockIdx.y;
    const int j = cols[wk];
    if (j < 0 || j >= n) return;                       // no accepted move: unchanged
    float *D = dinv + (size_t)wk * n * n;
    const float *r = rows + (size_t)wk * n;
    const float *w = work + (size_t)wk * 2 * n;
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    const bool kin = k < n;
    const int l0 = q * RPW;
    const int nr = max(0, min(RPW, n - l0));             // rows of this warp
    float d[RPW];
    float acc = 0.0f;
    {
        const float *pd = D + (size_t)l0 * n + (kin ? k : 0);
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            d[i] = (kin && i < nr) ? *pd : 0.0f;
            if (i < nr) acc = fmaf(__ldg(r + l0 + i), d[i], acc);
            pd += n;
        }
    }
    part[q][lane] = acc;
    __syncthreads();
    float wk_ = 0.0f;
#pragma unroll
    for (int p = 0; p < FU_WARPS; ++p) wk_ += part[p][lane];
    const float f = (wk_ - (k == j ? 1.0f : 0.0f)) / w[j];
    if (kin) {
        float *pd = D + (size_t)l0 * n + k;
        const float *cj = w + n + l0;
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            if (i < nr) *pd = fmaf(-cj[i], f, d[i]);
            pd += n;
        }
    }
}

template <int RPW>
void launch_fused(int n_walkers, int n, float *dinv, const float *rows, const int *cols,
                  float *work, cudaStream_t stream)
{
    sm_column_kernel<<<n_walkers, 32, 0, stream>>>(n, dinv, rows, cols, work);
    const dim3 g((n + 31) / 32, n_walkers);
    sm_fused_kernel<RPW><<<g, 32 * FU_WARPS, 0, stream>>>(n, dinv, rows, cols, work);
}

}  // namespace

cudaError_t launch_sm_update(int n_walkers, int n, float *dinv, const float *rows, const int *cols,
                             float *work, cudaStream_t stream)
{
    const int rpw = (n + FU_WARPS - 1) / FU_WARPS;
    if (rpw <= FU_MAX_ROWS) {
        if (rpw <= 16) launch_fused<16>(n_walkers, n, dinv, rows, cols, work, stream);
        else if (rpw <= 32) launch_fused<32>(n_walkers, n, dinv, rows, cols, work, stream);
        else if (rpw <= 48) launch_fused<48>(n_walkers, n, dinv, rows, cols, work, stream);
        else launch_fused<FU_MAX_ROWS>(n_walkers, n, dinv, rows, cols, work, stream);
        return cudaGetLastError();
    }
    const dim3 g1((n + 31) / 32, n_walkers);
    sm_gemv_kernel<<<g1, 32 * SM_PARTS, 0, stream>>>(n, dinv, rows, cols, work);
    const dim3 g2((n + SM_THREADS - 1) / SM_THREADS, (n + SM_ROWS - 1) / SM_ROWS, n_walkers);
    sm_rank1_kernel<<<g2, SM_THREADS, 0, stream>>>(n, dinv, cols, work);
    return cudaGetLastError();
}

}  // namespace blip
