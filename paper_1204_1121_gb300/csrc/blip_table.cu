// Table construction: the caller's coefficient table a[l, s~] (Eq. 7; layout
// [n1][n2][n3][Lreal], orbital index fastest, as in the paper's a[l,jx,jy,jz]
// with l sequential, Sec. II.B) is copied into the library's layout:
//
//   rows [n1][n2][n3 + 3][row_stride]: z-plane iz' stores the sites of plane
//   (iz' - 1) mod n3, so a stencil column's 4 sites i2-1 .. i2+2 are the 4
//   consecutive stored rows i2 .. i2+3 for every base plane i2 (three ghost
//   planes: iz' = 0, n3 + 1, n3 + 2).  Each row is padded with zeros to
//   row_stride elements (a whole number of 512-byte warp chunks).
//
// Quantised kinds (BF16 / FP16) store q = RN(a / s_l) with the per-component
// scale s_l = max over all sites of |a_l| (one shared scale per complex
// orbital), so |q| <= 1; the scale is applied once after accumulation.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "blip_internal.h"

namespace blip {

namespace {

template <typename S>
__global__ void stage_rows_kernel(const S *__restrict__ src, long long row0, long long nrows,
                                  int n2, int n3, int Lreal, long long row_stride,
                                  float *__restrict__ dst)
{
    const long long total = nrows * row_stride;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / row_stride;
        const int l = (int)(i - r * row_stride);
        const float v = l < Lreal ? (float)src[r * Lreal + l] : 0.0f;
        const long long R = row0 + r;
        const long long col = R / n3;                  // ix * n2 + iy
        const int iz = (int)(R - col * n3);
        const long long base = col * (long long)(n3 + 3);
        dst[(base + iz + 1) * row_stride + l] = v;
        if (iz == n3 - 1) dst[base * row_stride + l] = v;                    // plane -1
        if (iz == 0) dst[(base + n3 + 1) * row_stride + l] = v;              // plane n3
        if (iz == 1) dst[(base + n3 + 2) * row_stride + l] = v;              // plane n3 + 1
    }
}

__global__ void absmax_kernel(const float *__restrict__ t, long long rows, long long row_stride,
                              int Lreal, unsigned int *__restrict__ out)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= Lreal) return;
    float m = 0.0f;
    for (long long r = blockIdx.y; r < rows; r += gridDim.y)
        m = fmaxf(m, fabsf(t[r * row_stride + l]));
    atomicMax(out + l, __float_as_uint(m));   // non-negative floats order as their bits
}

__global__ void make_scales_kernel(const unsigned int *__restrict__ bits, int Lreal, int pairs,
                                   float *__restrict__ scales)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= Lreal) return;
    float s = __uint_as_float(bits[l]);
    if (pairs) s = fmaxf(__uint_as_float(bits[l ^ 1]), s);
    scales[l] = s > 0.0f ? s : 1.0f;
}

template <typename Q>
__device__ __forceinline__ Q to_q(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_q<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_q<__half>(float x) { return __float2half_rn(x); }

template <typename Q>
__global__ void quantize_kernel(const float *__restrict__ src, long long rows, long long row_stride,
                                int Lreal, const float *__restrict__ scales, Q *__restrict__ dst)
{
    const long long total = rows * row_stride;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(i % row_stride);
        const float v = l < Lreal ? src[i] / scales[l] : 0.0f;
        dst[i] = to_q<Q>(v);
    }
}

unsigned grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 65535LL * 32) b = 65535LL * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_stage_rows(const void *src, int src_is_double, long long row0, long long nrows,
                              const Geometry &geo, int Lreal, long long row_stride, float *dst,
                              cudaStream_t stream)
{
    const unsigned g = grid_for(nrows * row_stride, 256);
    if (src_is_double)
        stage_rows_kernel<double><<<g, 256, 0, stream>>>(static_cast<const double *>(src), row0,
                                                         nrows, geo.n[1], geo.n[2], Lreal,
                                                         row_stride, dst);
    else
        stage_rows_kernel<float><<<g, 256, 0, stream>>>(static_cast<const float *>(src), row0,
                                                        nrows, geo.n[1], geo.n[2], Lreal,
                                                        row_stride, dst);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const float *table, long long rows, long long row_stride, int Lreal,
                          unsigned int *absmax_bits, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(absmax_bits, 0, sizeof(unsigned int) * (size_t)Lreal, stream);
    if (e != cudaSuccess) return e;
    dim3 grid((Lreal + 127) / 128, (unsigned)(rows < 2048 ? rows : 2048));
    absmax_kernel<<<grid, 128, 0, stream>>>(table, rows, row_stride, Lreal, absmax_bits);
    return cudaGetLastError();
}

cudaError_t launch_make_scales(const unsigned int *absmax_bits, int Lreal, int pairs,
                               float *scales, cudaStream_t stream)
{
    make_scales_kernel<<<(Lreal + 255) / 256, 256, 0, stream>>>(absmax_bits, Lreal, pairs, scales);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float *src, long long rows, long long row_stride, int Lreal,
                            const float *scales, int elem, void *dst, cudaStream_t stream)
{
    const unsigned g = grid_for(rows * row_stride, 256);
    if (elem == ELEM_BF16)
        quantize_kernel<__nv_bfloat16><<<g, 256, 0, stream>>>(
            src, rows, row_stride, Lreal, scales, static_cast<__nv_bfloat16 *>(dst));
    else if (elem == ELEM_F16)
        quantize_kernel<__half><<<g, 256, 0, stream>>>(src, rows, row_stride, Lreal, scales,
                                                       static_cast<__half *>(dst));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// Read a buffer larger than L2 through L2 (no writes), so that L2 holds
// only clean lines of it afterwards: the autotuner's cold start for each
// timed run.
__global__ void l2_sweep_kernel(const uint4 *__restrict__ buf, long long n, int *__restrict__ sink)
{
    unsigned acc = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint4 v = __ldcg(buf + i);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    // sink is null at every launch, but the compiler cannot know it: the
    // loads stay in the program.
    if (sink != nullptr && acc == 0x9e3779b9u) *sink = (int)acc;
}

// Read a buffer reps times through L2 (L1 bypassed): with a buffer that fits
// in L2 after the first pass, the L2 -> SM read bandwidth.
__global__ void l2_read_kernel(const uint4 *__restrict__ buf, long long n, int reps,
                               int *__restrict__ sink)
{
    unsigned acc = 0;
    for (int r = 0; r < reps; ++r)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const uint4 v = __ldcg(buf + i);
            acc = __funnelshift_l(acc, acc, 1) ^ v.x ^ v.y ^ v.z ^ v.w;
        }
    // sink is null at every launch, but the compiler cannot know it: the
    // loads stay in the program.
    if (sink != nullptr && acc == 0x9e3779b9u) *sink = (int)acc;
}

cudaError_t launch_l2_read(const void *buf, size_t bytes, int reps, int sm_count,
                           cudaStream_t stream)
{
    l2_read_kernel<<<4 * sm_count, 512, 0, stream>>>(static_cast<const uint4 *>(buf),
                                                     (long long)(bytes / 16), reps, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_l2_sweep(const void *buf, size_t bytes, int sm_count, cudaStream_t stream)
{
    l2_sweep_kernel<<<4 * sm_count, 512, 0, stream>>>(static_cast<const uint4 *>(buf),
                                                      (long long)(bytes / 16), nullptr);
    return cudaGetLastError();
}

}  // namespace blip
