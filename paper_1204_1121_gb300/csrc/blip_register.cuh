// Register-gather evaluation kernel (template; instantiated per element type
// and chunk count in blip_reg_*.cu): values, gradients and Laplacians of all orbitals at a
// batch of electron positions from a periodic cubic-blip table.
//
// Math (Uejima & Maezono, Sec. II.B): psi_l(r) = sum over the 64 sites of the
// 4 x 4 x 4 stencil around r (Eq. 7) of a_{l,s} Theta_s(r) (Eq. 11.12.24.1),
// Theta_s = product of three 1-D cubic B-splines of the grid-coordinate
// distances (Eq. 11.12.24.2).  Gradient and Laplacian follow by the chain rule
// with J = diag(n) A^{-1}: grad = J^T grad_g, lap = sum_ab (J J^T)_ab d_a d_b.
//
// Work decomposition (GB300-first, not the paper's thread mapping): one warp
// evaluates one electron for 1-3 "chunks" of 32 lanes x one 16-byte vector of
// orbital components, so a stencil row is read with fully coalesced 128-bit
// loads along the orbital index (the orbital-contiguous layout the paper uses
// for coalescing, Sec. IV.B).  The warp itself
//   1. wraps the position into the cell and finds the base cell in FP64
//      (lanes 0-2, one lattice direction each),
//   2. forms the 64 x 5 combined weights (value, Cartesian gradient,
//      Laplacian) in FP32, two stencil sites per lane, into its own slice of
//      shared memory, together with the 16 stencil-column row indices,
//   3. contracts: for each of the 16 columns, 4 z-contiguous rows (the table
//      stores three ghost planes along a_3 so the 4 rows of a column never
//      wrap) x 5 FMAs per component,
//   4. scales (quantised tables) and writes the five outputs with streaming
//      stores at the electron's original index.
// No block-level synchronisation is needed: each warp owns its shared slice.
#pragma once

#include <type_traits>

#include "blip_device.cuh"

namespace blip {
namespace reg {

using namespace dev;

template <int CPW, int VEC, bool VONLY, int GEO>
__device__ __forceinline__ void store_outputs(const EvalParams &p, int e, int grp, int lane,
                                              float (&acc)[CPW][VONLY ? 1 : 5][VEC],
                                              const WarpSlice &ws)
{
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
        const int chunk = grp * CPW + c;
        if (chunk >= p.nchunk) break;                    // warp-uniform
        store_chunk<VEC, VONLY, GEO == 1>(p, e, chunk, lane, acc[c], ws.phase);
    }
}

// Contract RB rows (stencil sites pt0 .. pt0 + RB - 1) held in registers
// into the accumulators: 5 FMAs per component per row.
template <typename T, int CPW, int VEC, bool VONLY, int RB>
__device__ __forceinline__ void contract_rows(const WarpSlice &ws, int pt0,
                                              const uint4 (&buf)[RB][CPW],
                                              float (&acc)[CPW][VONLY ? 1 : 5][VEC],
                                              AccPairs<VEC> (&a5)[CPW])
{
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const float4 w = ws.w4[pt0 + r];
        const float wl = VONLY ? 0.0f : ws.wl[pt0 + r];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
            float f[VEC];
            Elt<T>::unpack(buf[r][c], f);
            if constexpr (VONLY) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[c][0][v] = fmaf(w.x, f[v], acc[c][0][v]);
            } else {
                pairs_fma(a5[c], w, wl, f);
            }
        }
    }
}

template <bool L1ALLOC>
__device__ __forceinline__ uint4 load_row(const void *p)
{
    if constexpr (L1ALLOC) return ldg_shared_rows(p);
    else return ldg_stream(p);
}

// Register-gather kernel: each lane loads its 16-byte slices of the 64 rows
// straight into registers (4 columns = 16 rows in flight per batch for one
// chunk, fewer for more chunks).
// GEO: 0 = FP64 wrap in the kernel, 1 = FP64 wrap + Bloch phases, 2 = per-slot
// geometry records from the sort pre-pass.
template <typename T, int CPW, bool VONLY, int PIPE, int GEO>
__global__ void __launch_bounds__(512) blip_eval_register(EvalParams p)
{
    constexpr int VEC = Elt<T>::VEC;
    constexpr int NW = VONLY ? 1 : 5;
    constexpr int COLS = CPW == 1 ? 4 : (CPW == 2 ? 2 : 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSlice &ws = reinterpret_cast<WarpSlice *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;

    check_offsets(p);

    const long long wpb = blockDim.x >> 5;
    const long long nwarps = (long long)gridDim.x * wpb;
    const char *tbase = reinterpret_cast<const char *>(p.table);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);

    // PIPE == 3: the warps of a block take consecutive electrons for the same
    // chunk group, so in a sorted batch they share stencil rows through L1
    // PIPE == 4: as 3, and the warps of a block step through the row batches
    // in lockstep (a block barrier per batch), so a row one warp brings into
    // L1 is still there when its neighbours ask for it
    constexpr bool BLOCKED = PIPE == 3 || PIPE == 4;
    const long long total = BLOCKED
        ? (long long)((p.n_elec + wpb - 1) / wpb) * p.groups * wpb : p.items;
    for (long long item = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); item < total;
         item += nwarps) {
        int slot, grp;
        bool dummy = false;          // PIPE 4: a padding warp that keeps the block in step
        if constexpr (BLOCKED) {
            const long long blk = item / wpb;
            const long long eb = blk / p.groups;
            grp = (int)(blk - eb * p.groups);
            slot = (int)(eb * wpb + (item - blk * wpb));
            if (slot >= p.n_elec) {                          // warp-uniform
                if constexpr (PIPE == 3) continue;
                dummy = true;
                slot = p.n_elec - 1;
            }
        } else if (p.group_major) {
            // every electron's first chunk group, then the second, ...: the
            // warps in flight cover more electrons with a smaller slice of
            // each row, so more of the rows they share stay in L2
            grp = (int)(item / p.n_elec);
            slot = (int)(item - (long long)grp * p.n_elec);
        } else {
            slot = (int)(item / p.groups);
            grp = (int)(item - (long long)slot * p.groups);
        }
        const int e = p.perm ? p.perm[slot] : slot;

        float acc[CPW][NW][VEC];
#pragma unroll
        for (int c = 0; c < CPW; ++c)
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[c][k][v] = 0.0f;
        AccPairs<VEC> a5[CPW];         // five-output accumulators (unused for values only)
#pragma unroll
        for (int c = 0; c < CPW; ++c) pairs_zero(a5[c]);

        __syncwarp();                      // previous item's readers are done with the slice
        float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f;
        constexpr bool EARLY = PIPE == 1 || PIPE == 3 || PIPE == 4 || PIPE == 5;   // first loads before the weights
        const int bad = EARLY ? stencil_geometry_warp<GEO>(p, e, lane, ws, t0, t1, t2, slot)
                              : stencil_setup_warp<GEO>(p, e, lane, ws, slot);
        if (bad && lane == 0 && !dummy) atomicOr(p.status, bad);
        if (bad & BLIP_STATUS_NONFINITE_POS) {
            if constexpr (PIPE == 4) {
                // stay in step with the block: contract harmless rows, store NaN
                if (lane < 16) ws.colrow[lane] = 0;
                t0 = t1 = t2 = 0.0f;
                __syncwarp();
            } else {
#pragma unroll
                for (int c = 0; c < CPW; ++c)
#pragma unroll
                    for (int k = 0; k < NW; ++k)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[c][k][v] = __int_as_float(0x7fc00000);
                store_outputs<CPW, VEC, VONLY, GEO>(p, e, grp, lane, acc, ws);
                continue;
            }
        }

        size_t coff[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
            const int chunk = min(grp * CPW + c, p.nchunk - 1);   // clamp: in-bounds duplicate
            coff[c] = ((size_t)chunk * 32 * VEC + (size_t)lane * VEC) * sizeof(T);
        }

        if constexpr (PIPE == 2) {
            // software-pipelined with a rolled loop over pairs of batches
            // (smaller code: the fully unrolled form misses in the instruction
            // cache when three chunks are in flight)
            constexpr int RB = CPW == 1 ? 4 : (CPW == 2 ? 2 : 1);
            constexpr int NB = 64 / RB;
            uint4 b0[RB][CPW], b1[RB][CPW];
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const char *rp = tbase + (size_t)(ws.colrow[r >> 2] + (r & 3)) * rowb;
#pragma unroll
                for (int c = 0; c < CPW; ++c) b0[r][c] = ldg_stream(rp + coff[c]);
            }
#pragma unroll 1
            for (int b = 0; b < NB; b += 2) {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int pt = (b + 1) * RB + r;
                    const char *rp = tbase + (size_t)(ws.colrow[pt >> 2] + (pt & 3)) * rowb;
#pragma unroll
                    for (int c = 0; c < CPW; ++c) b1[r][c] = ldg_stream(rp + coff[c]);
                }
                contract_rows<T, CPW, VEC, VONLY, RB>(ws, b * RB, b0, acc, a5);
                if (b + 2 < NB) {
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const int pt = (b + 2) * RB + r;
                        const char *rp = tbase + (size_t)(ws.colrow[pt >> 2] + (pt & 3)) * rowb;
#pragma unroll
                        for (int c = 0; c < CPW; ++c) b0[r][c] = ldg_stream(rp + coff[c]);
                    }
                }
                contract_rows<T, CPW, VEC, VONLY, RB>(ws, (b + 1) * RB, b1, acc, a5);
            }
        } else if constexpr (PIPE == 1 || PIPE == 3 || PIPE == 4 || PIPE == 5) {
            // software-pipelined: the next batch of RB rows (PIPE 5: the next
            // two batches) is in flight while the current batch is contracted
            constexpr int RB = CPW == 1 ? 8 : (CPW == 2 ? 4 : 2);
            constexpr int NB = 64 / RB;
            constexpr int NBUF = PIPE == 5 ? 3 : 2;
            uint4 buf[NBUF][RB][CPW];
#pragma unroll
            for (int q = 0; q < NBUF - 1; ++q)
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int pt = q * RB + r;
                    const char *rp = tbase + (size_t)(ws.colrow[pt >> 2] + (pt & 3)) * rowb;
#pragma unroll
                    for (int c = 0; c < CPW; ++c) buf[q][r][c] = load_row<BLOCKED>(rp + coff[c]);
                }
            stencil_weights_warp(p, t0, t1, t2, lane, ws);   // overlaps the first loads
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if constexpr (PIPE == 4) __syncthreads();
                if (b + NBUF - 1 < NB) {
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const int pt = (b + NBUF - 1) * RB + r;
                        const char *rp = tbase + (size_t)(ws.colrow[pt >> 2] + (pt & 3)) * rowb;
#pragma unroll
                        for (int c = 0; c < CPW; ++c)
                            buf[(b + NBUF - 1) % NBUF][r][c] = load_row<BLOCKED>(rp + coff[c]);
                    }
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int pt = b * RB + r;
                    const float4 w = ws.w4[pt];
                    const float wl = VONLY ? 0.0f : ws.wl[pt];
#pragma unroll
                    for (int c = 0; c < CPW; ++c) {
                        float f[VEC];
                        Elt<T>::unpack(buf[b % NBUF][r][c], f);
                        if constexpr (VONLY) {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[c][0][v] = fmaf(w.x, f[v], acc[c][0][v]);
                        } else {
                            pairs_fma(a5[c], w, wl, f);
                        }
                    }
                }
            }
        } else {
    #pragma unroll 1
            for (int c0 = 0; c0 < 16; c0 += COLS) {
                uint4 raw[COLS][4][CPW];
    #pragma unroll
                for (int cc = 0; cc < COLS; ++cc) {
                    const char *rp = tbase + (size_t)ws.colrow[c0 + cc] * rowb;
    #pragma unroll
                    for (int kz = 0; kz < 4; ++kz)
    #pragma unroll
                        for (int c = 0; c < CPW; ++c)
                            raw[cc][kz][c] = ldg_stream(rp + kz * rowb + coff[c]);
                }
    #pragma unroll
                for (int cc = 0; cc < COLS; ++cc)
    #pragma unroll
                    for (int kz = 0; kz < 4; ++kz) {
                        const int pt = (c0 + cc) * 4 + kz;
                        const float4 w = ws.w4[pt];
                        const float wl = VONLY ? 0.0f : ws.wl[pt];
    #pragma unroll
                        for (int c = 0; c < CPW; ++c) {
                            float f[VEC];
                            Elt<T>::unpack(raw[cc][kz][c], f);
                                if constexpr (VONLY) {
#pragma unroll
                                for (int v = 0; v < VEC; ++v)
                                    acc[c][0][v] = fmaf(w.x, f[v], acc[c][0][v]);
                            } else {
                                pairs_fma(a5[c], w, wl, f);
                            }
                        }
                    }
            }
        }
        if constexpr (!VONLY) {
#pragma unroll
            for (int c = 0; c < CPW; ++c) pairs_out(a5[c], acc[c]);
        }
        if constexpr (PIPE == 4) {
            if (dummy) continue;
            if (bad & BLIP_STATUS_NONFINITE_POS) {
#pragma unroll
                for (int c = 0; c < CPW; ++c)
#pragma unroll
                    for (int k = 0; k < NW; ++k)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[c][k][v] = __int_as_float(0x7fc00000);
            }
        }
        store_outputs<CPW, VEC, VONLY, GEO>(p, e, grp, lane, acc, ws);
    }
}

template <typename T, int CPW, bool VONLY, int GEO>
void launch_pipe(const EvalParams &p, int pipe, dim3 g, dim3 b, size_t smem, cudaStream_t stream)
{
    if (pipe == 5) {
        // three row buffers only fit the registers for one FP32 chunk
        if constexpr (std::is_same<T, float>::value && CPW == 1)
            blip_eval_register<T, CPW, VONLY, 5, GEO><<<g, b, smem, stream>>>(p);
    } else if (pipe == 4) blip_eval_register<T, CPW, VONLY, 4, GEO><<<g, b, smem, stream>>>(p);
    else if (pipe == 3) blip_eval_register<T, CPW, VONLY, 3, GEO><<<g, b, smem, stream>>>(p);
    else if (pipe == 2) blip_eval_register<T, CPW, VONLY, 2, GEO><<<g, b, smem, stream>>>(p);
    else if (pipe == 1) blip_eval_register<T, CPW, VONLY, 1, GEO><<<g, b, smem, stream>>>(p);
    else blip_eval_register<T, CPW, VONLY, 0, GEO><<<g, b, smem, stream>>>(p);
}

template <typename T, int CPW, bool VONLY>
cudaError_t launch_register_t(const EvalParams &p, int warps, int pipe, cudaStream_t stream)
{
    const size_t smem = sizeof(WarpSlice) * (size_t)warps;
    long long blocks = (p.items + warps - 1) / warps;
    if (blocks < 1) blocks = 1;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    if (pipe >= 3) {                 // whole blocks of consecutive electrons per chunk group
        blocks = (long long)((p.n_elec + warps - 1) / warps) * p.groups;
        if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    }
    const dim3 g((unsigned)blocks), b(32 * warps);
    if (p.n_k) {
        if constexpr (std::is_same<T, __half>::value) {
            return cudaErrorInvalidValue;              // FP16 storage is real only
        } else {
            launch_pipe<T, CPW, VONLY, 1>(p, pipe, g, b, smem, stream);
        }
    } else if (p.georec) {
        launch_pipe<T, CPW, VONLY, 2>(p, pipe, g, b, smem, stream);
    } else {
        launch_pipe<T, CPW, VONLY, 0>(p, pipe, g, b, smem, stream);
    }
    return cudaGetLastError();
}

template <typename T, int CPW>
cudaError_t launch_register_vo(const EvalParams &p, int warps, int pipe, cudaStream_t stream)
{
    if (p.grads) return launch_register_t<T, CPW, false>(p, warps, pipe, stream);
    return launch_register_t<T, CPW, true>(p, warps, pipe, stream);
}

}  // namespace reg
}  // namespace blip
