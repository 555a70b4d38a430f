// Cell-grouped evaluation kernel for dense batches: electrons that fall in the
// same grid cell have the same 64 stencil rows (Eq. 7), so one load of a row
// can feed all of them.  After the spatial sort the electrons of one cell sit
// in consecutive slots; the warp whose slot starts a group of up to G such
// electrons forms G weight sets and, for each of the 64 rows, loads its
// 16-byte slice once and does 5 FMAs per component for every member of the
// group.  Warps whose slot is not a group leader return at once.  Each
// output is still the same fixed-order 64-term sum as in the other kernels,
// so results are bitwise identical to them.
#include <type_traits>

#include "blip_device.cuh"

namespace blip {

namespace {

using namespace dev;

template <typename T, int G, bool VONLY, int GEO>
__global__ void __launch_bounds__(256) blip_eval_grouped(EvalParams p, const int *keys,
                                                         const int *cell_end)
{
    constexpr int VEC = Elt<T>::VEC;
    constexpr int NW = VONLY ? 1 : 5;
    constexpr int RB = 4;                          // rows per pipelined batch
    constexpr int NB = 64 / RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSlice *ws = reinterpret_cast<WarpSlice *>(smem_raw) + (threadIdx.x >> 5) * G;
    const int lane = threadIdx.x & 31;
    check_offsets(p);
    const long long wpb = blockDim.x >> 5;
    const long long nwarps = (long long)gridDim.x * wpb;
    const char *tbase = reinterpret_cast<const char *>(p.table);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);

    for (long long item = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); item < p.items;
         item += nwarps) {
        const int slot = (int)(item / p.nchunk);
        const int chunk = (int)(item - (long long)slot * p.nchunk);
        const int key = keys[p.perm[slot]];
        const int start = key ? cell_end[key - 1] : 0;
        if ((slot - start) % G != 0) continue;              // not a group leader
        const int gn = min(G, cell_end[key] - slot);
        int e[G], bad[G];
#pragma unroll
        for (int m = 0; m < G; ++m) {
            e[m] = 0;
            bad[m] = 0;
            if (m < gn) {
                e[m] = p.perm[slot + m];
                __syncwarp();
                bad[m] = stencil_setup_warp<GEO>(p, e[m], lane, ws[m], slot + m);
                if (bad[m] && lane == 0 && chunk == 0) atomicOr(p.status, bad[m]);
            }
        }
        float acc[G][NW][VEC];
#pragma unroll
        for (int m = 0; m < G; ++m)
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[m][k][v] = 0.0f;
        // members share the cell, so they share the rows; a cell-less
        // position (key of the last bucket) has none and gives NaN
        if (!(bad[0] & BLIP_STATUS_NONFINITE_POS)) {
            const size_t coff = ((size_t)chunk * 32 * VEC + (size_t)lane * VEC) * sizeof(T);
            uint4 b0[RB], b1[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r)
                b0[r] = ldg_stream(tbase + (size_t)(ws[0].colrow[r >> 2] + (r & 3)) * rowb + coff);
#pragma unroll 1
            for (int b = 0; b < NB; b += 2) {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int pt = (b + 1) * RB + r;
                    b1[r] = ldg_stream(tbase + (size_t)(ws[0].colrow[pt >> 2] + (pt & 3)) * rowb + coff);
                }
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    if (half == 1 && b + 2 < NB) {
#pragma unroll
                        for (int r = 0; r < RB; ++r) {
                            const int pt = (b + 2) * RB + r;
                            b0[r] = ldg_stream(tbase + (size_t)(ws[0].colrow[pt >> 2] + (pt & 3)) * rowb
                                               + coff);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const int pt = (b + half) * RB + r;
                        float f[VEC];
                        Elt<T>::unpack(half == 0 ? b0[r] : b1[r], f);
#pragma unroll
                        for (int m = 0; m < G; ++m) {
                            if (m < gn) {
                                const float4 w = ws[m].w4[pt];
                                const float wl = VONLY ? 0.0f : ws[m].wl[pt];
#pragma unroll
                                for (int v = 0; v < VEC; ++v) {
                                    acc[m][0][v] = fmaf(w.x, f[v], acc[m][0][v]);
                                    if constexpr (!VONLY) {
                                        acc[m][1][v] = fmaf(w.y, f[v], acc[m][1][v]);
                                        acc[m][2][v] = fmaf(w.z, f[v], acc[m][2][v]);
                                        acc[m][3][v] = fmaf(w.w, f[v], acc[m][3][v]);
                                        acc[m][4][v] = fmaf(wl, f[v], acc[m][4][v]);
                                    }
                                }
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < G; ++m) {
            if (m < gn) {
                if (bad[m] & BLIP_STATUS_NONFINITE_POS) {
#pragma unroll
                    for (int k = 0; k < NW; ++k)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[m][k][v] = __int_as_float(0x7fc00000);
                }
                store_chunk<VEC, VONLY, GEO == 1>(p, e[m], chunk, lane, acc[m], ws[m].phase);
            }
        }
    }
}

// Raise one instantiation's dynamic shared-memory cap once (8 warps x 4
// slices pass the 48 KB default).
template <typename K>
cudaError_t allow_smem(K kernel, size_t smem, bool &done)
{
    if (done || smem <= 48 * 1024) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T, int G, bool VONLY>
cudaError_t launch_grouped_t(const EvalParams &p, int warps, const int *keys, const int *cell_end,
                             cudaStream_t stream)
{
    const size_t smem = sizeof(WarpSlice) * (size_t)warps * G;
    static bool done[3] = {false, false, false};
    cudaError_t e = cudaSuccess;
    if (p.n_k) {
        if constexpr (!std::is_same<T, __half>::value)
            e = allow_smem(blip_eval_grouped<T, G, VONLY, 1>, smem, done[1]);
    } else if (p.georec) {
        e = allow_smem(blip_eval_grouped<T, G, VONLY, 2>, smem, done[2]);
    } else {
        e = allow_smem(blip_eval_grouped<T, G, VONLY, 0>, smem, done[0]);
    }
    if (e != cudaSuccess) return e;
    long long blocks = (p.items + warps - 1) / warps;
    if (blocks < 1) blocks = 1;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    if (p.n_k) {
        if constexpr (std::is_same<T, __half>::value) {
            return cudaErrorInvalidValue;              // FP16 storage is real only
        } else {
            blip_eval_grouped<T, G, VONLY, 1><<<(unsigned)blocks, 32 * warps, smem, stream>>>(
                p, keys, cell_end);
        }
    } else if (p.georec) {
        blip_eval_grouped<T, G, VONLY, 2><<<(unsigned)blocks, 32 * warps, smem, stream>>>(
            p, keys, cell_end);
    } else {
        blip_eval_grouped<T, G, VONLY, 0><<<(unsigned)blocks, 32 * warps, smem, stream>>>(
            p, keys, cell_end);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grouped_e(const EvalParams &p, int group, int warps, const int *keys,
                             const int *cell_end, cudaStream_t stream)
{
    const bool vo = p.grads == nullptr;
    if (group == 2)
        return vo ? launch_grouped_t<T, 2, true>(p, warps, keys, cell_end, stream)
                  : launch_grouped_t<T, 2, false>(p, warps, keys, cell_end, stream);
    if (group == 4)
        return vo ? launch_grouped_t<T, 4, true>(p, warps, keys, cell_end, stream)
                  : launch_grouped_t<T, 4, false>(p, warps, keys, cell_end, stream);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_grouped(const EvalParams &p, int elem, int group, int warps, const int *keys,
                           const int *cell_end, cudaStream_t stream)
{
    if (!p.perm || warps < 1 || warps > 8) return cudaErrorInvalidValue;
    switch (elem) {
    case ELEM_F32: return launch_grouped_e<float>(p, group, warps, keys, cell_end, stream);
    case ELEM_BF16: return launch_grouped_e<__nv_bfloat16>(p, group, warps, keys, cell_end, stream);
    case ELEM_F16: return launch_grouped_e<__half>(p, group, warps, keys, cell_end, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip
