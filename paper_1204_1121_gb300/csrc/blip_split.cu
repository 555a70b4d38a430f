// Split-stencil evaluation kernel for small, latency-bound launches: a few
// hundred electrons, or one electron at a time (the paper's particle-by-
// particle mode).  Same result as the other kernels up to the order of the
// 64-term sum (Eq. 11.12.24.1 with value, gradient and Laplacian).
//
// With few electrons in a launch, a register-gather warp spends its time
// waiting for its 64 stencil rows in a chain of a few batches.  Here a block
// of 4 warps takes one (electron, 512-byte chunk of components) item, and
// warp q takes the 16 sites of one a_1 slab (kx = q): it issues all 16 row
// loads at once, forms its 16 combined weights while they are in flight,
// contracts them, and the four partial sums are added in a fixed order
// (((q0 + q1) + q2) + q3) through shared memory.  One round of memory
// latency per item instead of several.  Deterministic; the summation order
// differs from the single-warp kernels, so the outputs agree with them to
// rounding, not bitwise.
#include "blip_device.cuh"

namespace blip {

namespace {

using namespace dev;

constexpr int kParts = 4;   // warps per item: one a_1 slab of 16 sites each

template <int VEC>
struct SplitSmem {
    float4 w4[kParts][16];
    float wl[kParts][16];
    float part[kParts - 1][5][VEC][32];   // partial sums of warps 1..3, lane fastest
};

template <typename T, bool VONLY, int GEO>
__global__ void __launch_bounds__(32 * kParts) blip_eval_split(EvalParams p)
{
    constexpr int VEC = Elt<T>::VEC;
    constexpr int NW = VONLY ? 1 : 5;
    __shared__ SplitSmem<VEC> sm;
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    check_offsets(p);
    const char *tbase = reinterpret_cast<const char *>(p.table);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);

    for (long long item = blockIdx.x; item < p.items; item += gridDim.x) {
        const int slot = (int)(item / p.nchunk);
        const int chunk = (int)(item - (long long)slot * p.nchunk);
        const int e = p.perm ? p.perm[slot] : slot;
        // geometry: every warp reduces the position itself (FP64 on lanes
        // 0-2), or reads the sort's record
        int i0, i1, i2, bad;
        float t0, t1, t2;
        if constexpr (GEO == 2) {
            const int4 gi = *reinterpret_cast<const int4 *>(p.georec + slot);
            const float4 gt = *reinterpret_cast<const float4 *>(&p.georec[slot].t[0]);
            i0 = gi.x; i1 = gi.y; i2 = gi.z; bad = gi.w;
            t0 = gt.x; t1 = gt.y; t2 = gt.z;
        } else {
            int ia = 0;
            float ta = 0.0f;
            bad = 0;
            if (lane < 3) {
                const double *r = p.pos + 3 * (size_t)e;
                bad = wrap_axis(p.geo, lane, r[0], r[1], r[2], ia, ta);
            }
            bad = __reduce_or_sync(FULL, bad);
            i0 = __shfl_sync(FULL, ia, 0); i1 = __shfl_sync(FULL, ia, 1); i2 = __shfl_sync(FULL, ia, 2);
            t0 = __shfl_sync(FULL, ta, 0); t1 = __shfl_sync(FULL, ta, 1); t2 = __shfl_sync(FULL, ta, 2);
        }
        if (bad && q == 0 && lane == 0 && chunk == 0) atomicOr(p.status, bad);
        const bool nan_pos = (bad & BLIP_STATUS_NONFINITE_POS) != 0;   // block-uniform

        float acc[NW][VEC];
        if (!nan_pos) {
            const size_t coff = ((size_t)chunk * 32 * VEC + (size_t)lane * VEC) * sizeof(T);
            // this warp's 16 rows: columns (kx = q, ky = 0..3), 4 stored rows each
            uint4 raw[16];
#pragma unroll
            for (int ky = 0; ky < 4; ++ky) {
                const char *rp = tbase + (size_t)column_row(p.geo, i0, i1, i2, 4 * q + ky) * rowb + coff;
#pragma unroll
                for (int kz = 0; kz < 4; ++kz) raw[4 * ky + kz] = ldg_stream(rp + kz * rowb);
            }
            // the slab's 16 combined weights while the rows are in flight
            if (lane < 16) site_weights(p.geo, t0, t1, t2, 16 * q + lane, sm.w4[q][lane], sm.wl[q][lane]);
            __syncwarp();
            AccPairs<VEC> ap;
            pairs_zero(ap);
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[k][v] = 0.0f;
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const float4 w = sm.w4[q][s];
                float f[VEC];
                Elt<T>::unpack(raw[s], f);
                if constexpr (VONLY) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[0][v] = fmaf(w.x, f[v], acc[0][v]);
                } else {
                    pairs_fma(ap, w, sm.wl[q][s], f);
                }
            }
            if constexpr (!VONLY) pairs_out(ap, acc);
        } else {
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[k][v] = __int_as_float(0x7fc00000);
        }
        if (q > 0) {
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) sm.part[q - 1][k][v][lane] = acc[k][v];
        }
        __syncthreads();
        if (q == 0) {
#pragma unroll
            for (int r = 0; r < kParts - 1; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[k][v] += sm.part[r][k][v][lane];
            store_chunk<VEC, VONLY>(p, e, chunk, lane, acc);
        }
        __syncthreads();   // the shared partials and weights are reused by the next item
    }
}

template <typename T, bool VONLY>
cudaError_t launch_split_t(const EvalParams &p, cudaStream_t stream)
{
    long long blocks = p.items;
    if (blocks < 1) blocks = 1;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    if (p.georec)
        blip_eval_split<T, VONLY, 2><<<(unsigned)blocks, 32 * kParts, 0, stream>>>(p);
    else
        blip_eval_split<T, VONLY, 0><<<(unsigned)blocks, 32 * kParts, 0, stream>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_split_elem(const EvalParams &p, cudaStream_t stream)
{
    if (p.grads) return launch_split_t<T, false>(p, stream);
    return launch_split_t<T, true>(p, stream);
}

}  // namespace

cudaError_t launch_split(const EvalParams &p, int elem, cudaStream_t stream)
{
    if (p.n_k || p.groups != p.nchunk) return cudaErrorInvalidValue;   // one chunk per item
    switch (elem) {
    case ELEM_F32: return launch_split_elem<float>(p, stream);
    case ELEM_BF16: return launch_split_elem<__nv_bfloat16>(p, stream);
    case ELEM_F16: return launch_split_elem<__half>(p, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip
