// Fused quasi-simultaneous ratio kernel: the orbital evaluation of
// Eq. 11.12.24.1 contracted on the fly with one column of the inverse Slater
// matrix, so that only five numbers per electron leave the chip.
//
// For the trial move r'_j of electron j (Sec. IV.A, Eq. 11.12.23.1) the
// determinant ratio of the quasi-simultaneous update is
//     xi_j = sum_l psi_l(r'_j) (D^{-1})_{lj}
// (the new row of D dotted with column j of its inverse, the matrix-
// determinant lemma behind the Sherman-Morrison update of Sec. VI.D), and the
// drift and kinetic terms of the local energy need the same contraction of
// the gradient and Laplacian.  The kernel therefore writes, per electron,
//     ratio[j][0] = sum_l psi_l c_jl,  ratio[j][1..3] = sum_l grad psi_l c_jl,
//     ratio[j][4] = sum_l lap psi_l c_jl,
// with c_j the caller's column (D^{-1})_{. j} of the electron's own walker and
// spin, stored contiguously per electron.  Optionally the new row psi_l(r'_j)
// is written too (needed to update D^{-1} if the move is accepted).
//
// One warp per electron: the weights are formed once, then the warp walks the
// orbital chunks (32 lanes x 16 bytes each) with the software-pipelined
// 64-row gather, folds each chunk into five per-lane dot products, and ends
// with a fixed-order butterfly reduction (deterministic, no atomics).
#include "blip_device.cuh"

namespace blip {

namespace {

using namespace dev;

template <typename T, int GEO>
__global__ void __launch_bounds__(256) blip_eval_ratio_kernel(EvalParams p, const float *cols,
                                                              float *ratio)
{
    constexpr int VEC = Elt<T>::VEC;
    constexpr int RB = 8;                 // rows per pipelined batch
    constexpr int NB = 64 / RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSlice &ws = reinterpret_cast<WarpSlice *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    check_offsets(p);
    const long long wpb = blockDim.x >> 5;
    const long long nwarps = (long long)gridDim.x * wpb;
    const char *tbase = reinterpret_cast<const char *>(p.table);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);
    const size_t L = (size_t)p.Lreal;

    for (long long slot = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); slot < p.n_elec;
         slot += nwarps) {
        const int e = p.perm ? p.perm[slot] : (int)slot;
        __syncwarp();
        const int bad = stencil_setup_warp<GEO>(p, e, lane, ws, (int)slot);
        if (bad && lane == 0) atomicOr(p.status, bad);
        float dot[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (bad & BLIP_STATUS_NONFINITE_POS) {
            if (lane < 5) ratio[(size_t)e * 5 + lane] = __int_as_float(0x7fc00000);
            if (p.values)
                for (size_t l = lane; l < L; l += 32)
                    p.values[(size_t)e * L + l] = __int_as_float(0x7fc00000);
            continue;
        }
        for (int chunk = 0; chunk < p.nchunk; ++chunk) {
            const size_t coff = ((size_t)chunk * 32 * VEC + (size_t)lane * VEC) * sizeof(T);
            AccPairs<VEC> accp;
            pairs_zero(accp);
            uint4 buf[2][RB];
#pragma unroll
            for (int r = 0; r < RB; ++r)
                buf[0][r] = ldg_stream(tbase + (size_t)(ws.colrow[r >> 2] + (r & 3)) * rowb + coff);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (b + 1 < NB) {
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const int pt = (b + 1) * RB + r;
                        buf[(b + 1) & 1][r] = ldg_stream(
                            tbase + (size_t)(ws.colrow[pt >> 2] + (pt & 3)) * rowb + coff);
                    }
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int pt = b * RB + r;
                    const float4 w = ws.w4[pt];
                    const float wl = ws.wl[pt];
                    float f[VEC];
                    Elt<T>::unpack(buf[b & 1][r], f);
                    pairs_fma(accp, w, wl, f);
                }
            }
            float acc[5][VEC];
            pairs_out(accp, acc);
            const int l0 = chunk * 32 * VEC + lane * VEC;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int l = l0 + v;
                if (l < p.Lreal) {
                    const float sc = p.scales ? p.scales[l] : 1.0f;
                    const float c = cols[(size_t)e * L + l];
#pragma unroll
                    for (int k = 0; k < 5; ++k) dot[k] = fmaf(acc[k][v] * sc, c, dot[k]);
                    if (p.values) __stcs(p.values + (size_t)e * L + l, acc[0][v] * sc);
                }
            }
        }
        // fixed-order butterfly: every lane ends with the same total
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dot[k] += __shfl_xor_sync(FULL, dot[k], o);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 5; ++k) ratio[(size_t)e * 5 + k] = dot[k];
        }
    }
}

template <typename T>
cudaError_t launch_ratio_t(const EvalParams &p, const float *cols, float *ratio, int warps,
                           cudaStream_t stream)
{
    const size_t smem = sizeof(WarpSlice) * (size_t)warps;
    long long blocks = ((long long)p.n_elec + warps - 1) / warps;
    if (blocks < 1) blocks = 1;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    if (p.georec)
        blip_eval_ratio_kernel<T, 2><<<(unsigned)blocks, 32 * warps, smem, stream>>>(p, cols, ratio);
    else
        blip_eval_ratio_kernel<T, 0><<<(unsigned)blocks, 32 * warps, smem, stream>>>(p, cols, ratio);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ratio(const EvalParams &p, int elem, const float *cols, float *ratio,
                         int warps, cudaStream_t stream)
{
    if (warps < 1 || warps > 8) return cudaErrorInvalidValue;
    switch (elem) {
    case ELEM_F32: return launch_ratio_t<float>(p, cols, ratio, warps, stream);
    case ELEM_BF16: return launch_ratio_t<__nv_bfloat16>(p, cols, ratio, warps, stream);
    case ELEM_F16: return launch_ratio_t<__half>(p, cols, ratio, warps, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip
