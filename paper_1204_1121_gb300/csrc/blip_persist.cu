// Persistent two-batch register-gather kernel (FP32 tables, one 512-byte
// chunk of components per warp): the arithmetic of the pipelined register
// kernel (Eq. 11.12.24.1 with value, gradient and Laplacian; the same FMA
// order, so bitwise equal outputs), with the start of each electron taken off
// the critical path.
//
// In the one-electron-per-warp kernels every warp begins with a serial chain
// that keeps none of its rows in flight: the position load, the FP64 wrap
// (a slow pipe on this part) and only then the first row loads.  Here a grid
// of resident warps walks the (electron, chunk) items with a stride; for
// each item a warp
//   * first starts a cp.async copy of the next item's position (or its sort
//     record, and its output index) into its shared slice, so the copy
//     flies with the item's row loads (issued from within the row loop it
//     made the compiler spill registers), and
//   * once the last row batch of the current item is issued and a batch
//     contracted (the slice's column rows are then free), runs the next
//     item's FP64 wrap and writes its column rows, offsets and status into
//     the slice,
// so the next item's first two batches go out as soon as the current item
// is stored.  Items are walked in 32-bit (major, minor) steps.  Not for
// Bloch tables: the phases of the next electron would overwrite the current
// one's before its store.
#include "blip_device.cuh"

namespace blip {

namespace {

using namespace dev;

// Per-warp shared memory: the usual slice, the prefetched source of the
// next item's geometry, and that geometry's warp-uniform results.
struct PersistSlice {
    WarpSlice ws;
    alignas(16) double pre[4];   // next position (GEO 0) or sort record (GEO 2)
    float nt[3];                 // next item's FP32 offsets
    int nbad;                    // next item's status bits
    int ne;                      // next item's output index
    int nperm;                   // perm[next slot], prefetched
    int dq, dr;                  // the warp's item stride, as (major, minor) steps
};

template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;"
                 :: "r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem), "n"(BYTES)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Items are (major, minor) pairs: (slot, chunk group), or (chunk group,
// slot) when ordered chunk group slowest.  The warp steps through them with
// a fixed stride (dq, dr) in 32-bit arithmetic.
struct ItemPos {
    int maj, mn;
};

__device__ __forceinline__ int minor_count(const EvalParams &p)
{
    return p.group_major ? p.n_elec : p.groups;
}

__device__ __forceinline__ int major_count(const EvalParams &p)
{
    return p.group_major ? p.groups : p.n_elec;
}

__device__ __forceinline__ ItemPos step_item(const EvalParams &p, ItemPos it, int dq, int dr)
{
    const int mod = minor_count(p);
    it.mn += dr;
    it.maj += dq;
    if (it.mn >= mod) {
        it.mn -= mod;
        it.maj += 1;
    }
    return it;
}

__device__ __forceinline__ int item_slot(const EvalParams &p, ItemPos it)
{
    return p.group_major ? it.mn : it.maj;
}

__device__ __forceinline__ int item_group(const EvalParams &p, ItemPos it)
{
    return p.group_major ? it.maj : it.mn;
}

// The next item's geometry into the slice: column rows (by
// stencil_geometry_warp) and offsets, status and output index (lane 0).
// src: its prefetched position or record in the slice, or nullptr to read
// them from global memory.
template <int GEO>
__device__ __forceinline__ void next_geometry(const EvalParams &p, PersistSlice &ps, int e,
                                              int slot, int lane, const void *src)
{
    float t0, t1, t2;
    const int bad = stencil_geometry_warp<GEO>(p, e, lane, ps.ws, t0, t1, t2, slot, src);
    if (lane == 0) {
        ps.nt[0] = t0;
        ps.nt[1] = t1;
        ps.nt[2] = t2;
        ps.nbad = bad;
        ps.ne = e;
    }
}

// PROBE: 0 evaluates; 1 and 2 are the measurement probe behind
// blip_probe_gather: the same geometry, row loads and item walk with the
// weights and the contraction left out (the loaded words are folded into one
// word per lane), and for 2 the five output slices stored as usual.
template <bool VONLY, int GEO, int PROBE = 0>
__global__ void __launch_bounds__(512) blip_eval_persist(EvalParams p)
{
    constexpr int VEC = 4;
    constexpr int NW = VONLY ? 1 : 5;
    constexpr int RB = 8, NB = 8, NBUF = 3;     // 8-row batches, two in flight
    constexpr int LAST_ISSUE = NB - NBUF;       // step that issues the last batch
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PersistSlice &ps = reinterpret_cast<PersistSlice *>(smem_raw)[threadIdx.x >> 5];
    WarpSlice &ws = ps.ws;
    const int lane = threadIdx.x & 31;

    check_offsets(p);

    const char *tbase = reinterpret_cast<const char *>(p.table);
    const size_t rowb = (size_t)p.row_stride * sizeof(float);
    // prefetch the next position only where its address is known early
    const bool pre_src = GEO == 2 || !p.perm;

    const long long first = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (first >= p.items) return;                 // warp-uniform
    {
        // the grid is at most one warp per item, so the stride fits 32 bits
        const int nw = gridDim.x * (blockDim.x >> 5);
        if (lane == 0) {
            ps.dq = nw / minor_count(p);
            ps.dr = nw - ps.dq * minor_count(p);
        }
    }
    ItemPos it{(int)(first / minor_count(p)), (int)(first % minor_count(p))};
    {
        const int slot = item_slot(p, it);
        next_geometry<GEO>(p, ps, p.perm ? p.perm[slot] : slot, slot, lane, nullptr);
    }
    for (;;) {
        __syncwarp();                             // the slice's next-item fields are written
        const int e = ps.ne, bad = ps.nbad;
        const float t0 = ps.nt[0], t1 = ps.nt[1], t2 = ps.nt[2];
        const int grp = item_group(p, it);
        if (bad && lane == 0) atomicOr(p.status, bad);

        float acc[NW][VEC];
        if (bad & BLIP_STATUS_NONFINITE_POS) {
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[k][v] = __int_as_float(0x7fc00000);
            store_chunk<VEC, VONLY>(p, e, grp, lane, acc);
            it = step_item(p, it, ps.dq, ps.dr);
            if (it.maj >= major_count(p)) break;
            const int slot = item_slot(p, it);
            __syncwarp();                         // every lane has read this item's fields
            next_geometry<GEO>(p, ps, p.perm ? p.perm[slot] : slot, slot, lane, nullptr);
            continue;
        }

#pragma unroll
        for (int k = 0; k < NW; ++k)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[k][v] = 0.0f;
        AccPairs<VEC> a5;
        pairs_zero(a5);
        unsigned fold = 0;                        // PROBE: the loaded words, folded
        {
            // the next item's source, into the slice while this item's rows fly
            const ItemPos nx = step_item(p, it, ps.dq, ps.dr);
            if (nx.maj < major_count(p)) {
                const int nslot = item_slot(p, nx);
                if constexpr (GEO == 2) {
                    if (lane < 2)
                        cp_async<16>(reinterpret_cast<char *>(ps.pre) + 16 * lane,
                                     reinterpret_cast<const char *>(p.georec + nslot) + 16 * lane);
                } else {
                    if (pre_src && lane < 3) cp_async<8>(&ps.pre[lane], p.pos + 3 * (size_t)nslot + lane);
                }
                if (p.perm && lane == 3) cp_async<4>(&ps.nperm, p.perm + nslot);
            }
        }
        const size_t coff = ((size_t)grp * 32 * VEC + (size_t)lane * VEC) * sizeof(float);
        uint4 buf[NBUF][RB];
#pragma unroll
        for (int q = 0; q < NBUF - 1; ++q)
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int pt = q * RB + r;
                buf[q][r] = ldg_stream(tbase + (size_t)(ws.colrow[pt >> 2] + (pt & 3)) * rowb + coff);
            }
        if constexpr (!PROBE) stencil_weights_warp(p, t0, t1, t2, lane, ws);   // overlaps the first loads
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b + NBUF - 1 < NB) {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int pt = (b + NBUF - 1) * RB + r;
                    buf[(b + NBUF - 1) % NBUF][r] =
                        ldg_stream(tbase + (size_t)(ws.colrow[pt >> 2] + (pt & 3)) * rowb + coff);
                }
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if constexpr (PROBE) {
                    const uint4 u = buf[b % NBUF][r];
                    fold ^= u.x ^ u.y ^ u.z ^ u.w;
                    continue;
                }
                const int pt = b * RB + r;
                const float4 w = ws.w4[pt];
                const float wl = VONLY ? 0.0f : ws.wl[pt];
                float f[VEC];
                Elt<float>::unpack(buf[b % NBUF][r], f);
                if constexpr (VONLY) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[0][v] = fmaf(w.x, f[v], acc[0][v]);
                } else {
                    pairs_fma(a5, w, wl, f);
                }
            }
            if (b == LAST_ISSUE) {
                // every row of this item is issued (and the batch contracted,
                // freeing its registers): the column rows may be replaced by
                // the next item's
                const ItemPos nx = step_item(p, it, ps.dq, ps.dr);
                if (nx.maj < major_count(p)) {
                    cp_async_wait_all();
                    __syncwarp();
                    const int nslot = item_slot(p, nx);
                    const int ne = p.perm ? ps.nperm : nslot;
                    next_geometry<GEO>(p, ps, ne, nslot, lane, pre_src ? ps.pre : nullptr);
                }
            }
        }
        if constexpr (PROBE == 1) {
            // no stores: the fold is written only under a condition the
            // compiler cannot decide (never true here: the probe passes no
            // outputs), so every load stays
            if (p.values && fold == 0x9e3779b9u) p.values[lane] = __uint_as_float(fold);
        } else if constexpr (PROBE == 2) {
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[k][v] = __uint_as_float(fold);
            store_chunk<VEC, VONLY>(p, e, grp, lane, acc);
        } else {
            if constexpr (!VONLY) pairs_out(a5, acc);
            store_chunk<VEC, VONLY>(p, e, grp, lane, acc);
        }
        it = step_item(p, it, ps.dq, ps.dr);
        if (it.maj >= major_count(p)) break;
        __syncwarp();                             // the weights are read by every lane
    }
}

template <bool VONLY, int GEO, int PROBE = 0>
cudaError_t launch_persist_t(const EvalParams &p, int warps, int sm_count, cudaStream_t stream)
{
    const size_t smem = sizeof(PersistSlice) * (size_t)warps;
    long long blocks = (p.items + warps - 1) / warps;
    // resident blocks per SM for this block size, once per configuration
    static int occ[17] = {0};
    if (occ[warps] == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, blip_eval_persist<VONLY, GEO, PROBE>,
                                                          32 * warps, smem) != cudaSuccess ||
            nb < 1)
            nb = 1;
        occ[warps] = nb;
    }
    const long long resident = (long long)occ[warps] * (sm_count > 0 ? sm_count : 1);
    if (blocks > resident) blocks = resident;
    if (blocks < 1) blocks = 1;
    blip_eval_persist<VONLY, GEO, PROBE><<<(unsigned)blocks, 32 * warps, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_persist(const EvalParams &p, int warps, int sm_count, cudaStream_t stream)
{
    if (p.n_k || p.groups != p.nchunk || warps < 1 || warps > 16) return cudaErrorInvalidValue;
    if (p.georec) {
        if (p.grads) return launch_persist_t<false, 2>(p, warps, sm_count, stream);
        return launch_persist_t<true, 2>(p, warps, sm_count, stream);
    }
    if (p.grads) return launch_persist_t<false, 0>(p, warps, sm_count, stream);
    return launch_persist_t<true, 0>(p, warps, sm_count, stream);
}

cudaError_t launch_probe(const EvalParams &p, int warps, int sm_count, bool store, cudaStream_t stream)
{
    if (p.n_k || p.georec || p.perm || p.groups != p.nchunk || warps < 1 || warps > 16)
        return cudaErrorInvalidValue;
    if (store) {
        if (!p.values || !p.grads || !p.laps) return cudaErrorInvalidValue;
        return launch_persist_t<false, 0, 2>(p, warps, sm_count, stream);
    }
    return launch_persist_t<false, 0, 1>(p, warps, sm_count, stream);
}

}  // namespace blip
