// Bulk-copy evaluation kernel: the same result as the register-gather kernel
// (Eq. 11.12.24.1 with value, gradient and Laplacian for every orbital), with
// the table reads moved off the registers onto the bulk-copy (TMA) engine.
//
// Persistent grid; each CTA is a producer/consumer pipeline over its items
// (item = electron x orbital tile of TW chunks; a chunk is 32 lanes x 16
// bytes of one row):
//   * producer warp: wraps the electron into the cell and finds its base
//     cell (FP64, lanes 0-2), then for each of the 16 stencil columns copies
//     the column's 4 consecutive stored rows (three ghost planes along a_3
//     keep them contiguous) restricted to the tile, with cp.async.bulk into a
//     ring of S shared-memory stages, signalling an mbarrier with the byte
//     count.  With one tile per row the 4 rows are one contiguous copy.
//   * TW consumer warps (one per chunk of the tile): wait for a stage, read
//     their 512-byte slice of each of the 4 rows, do 5 FMAs per component per
//     row with the combined weights (computed by each consumer warp from the
//     item's offsets, which the producer publishes beside the stage), release
//     the stage through a second mbarrier, and finally write the outputs.
// Every wait is bounded (about two seconds on the global timer); a wait that
// runs out sets BLIP_STATUS_TIMEOUT, the producer drains the copies it has in
// flight, and the CTA returns.
#include "blip_mbar.cuh"

namespace blip {

namespace {

using namespace dev;
using namespace mb;

struct ItemDesc {
    int e;        // electron index (after the optional sort permutation)
    int bad;      // status bits of its position
    float t[3];   // offsets from the base cell, FP32
    int pad[3];   // 32 bytes: keeps the weights that follow 16-byte aligned
};

struct BulkArgs {
    int tw;          // chunks per tile (= consumer warps)
    int ntiles;      // tiles per row
    int stages;      // ring depth S
    int stage_bytes; // 4 rows x tw x 512 bytes
    int stall;       // test hook: consumers never release the first stage
};

template <typename T, bool VONLY>
__global__ void __launch_bounds__(288) blip_eval_bulk(EvalParams p, BulkArgs b)
{
    constexpr int VEC = Elt<T>::VEC;
    constexpr int NW = VONLY ? 1 : 5;
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = b.stages;
    // layout: stages | full[S] | empty[S] | desc[S] | per-consumer weights
    unsigned char *stage0 = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * b.stage_bytes);
    uint64_t *empty = full + S;
    ItemDesc *desc = reinterpret_cast<ItemDesc *>(empty + S);
    WarpWeights *wts = reinterpret_cast<WarpWeights *>(desc + S);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncons = b.tw;
    check_offsets(p);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, ncons);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const long long items = (long long)p.n_elec * b.ntiles;
    const size_t row_bytes = (size_t)p.row_stride * sizeof(T);
    const char *tbase = reinterpret_cast<const char *>(p.table);

    if (warp == 0) {
        // ---------------- producer ----------------
        long long k = 0;           // stages issued
        bool ok = true;
        for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const int slot_e = (int)(it / b.ntiles);
            const int tile = (int)(it - (long long)slot_e * b.ntiles);
            const int e = p.perm ? p.perm[slot_e] : slot_e;
            int ia = 0, bad = 0;
            float ta = 0.0f;
            if (lane < 3) {
                const double *r = p.pos + 3 * (size_t)e;
                bad = wrap_axis(p.geo, lane, r[0], r[1], r[2], ia, ta);
            }
            bad = __reduce_or_sync(FULL, bad);
            const int i0 = __shfl_sync(FULL, ia, 0), i1 = __shfl_sync(FULL, ia, 1),
                      i2 = __shfl_sync(FULL, ia, 2);
            const float t0 = __shfl_sync(FULL, ta, 0), t1 = __shfl_sync(FULL, ta, 1),
                        t2 = __shfl_sync(FULL, ta, 2);
            const int crow = lane < 16 ? ((bad & BLIP_STATUS_NONFINITE_POS)
                                              ? 0 : column_row(p.geo, i0, i1, i2, lane))
                                       : 0;
            const int c0 = tile * b.tw;
            const int nc = min(b.tw, p.nchunk - c0);          // valid chunks in this tile
            const unsigned piece = (unsigned)nc * 512u;        // bytes per row in this tile
            for (int col = 0; col < 16; ++col) {
                const int row = __shfl_sync(FULL, crow, col);
                const int s = (int)(k % S);
                if (k >= S) {
                    const bool got = mbar_wait(empty + s, (unsigned)((k / S - 1) & 1));
                    if (!__all_sync(FULL, got)) {      // warp-uniform decision
                        ok = false;
                        break;
                    }
                }
                if (lane == 0) {
                    if (col == 0) {
                        ItemDesc d;
                        d.e = e; d.bad = bad; d.t[0] = t0; d.t[1] = t1; d.t[2] = t2;
                        d.pad[0] = d.pad[1] = d.pad[2] = 0;
                        desc[s] = d;
                    }
                    mbar_expect_tx(full + s, 4u * piece);
                    unsigned char *dst = stage0 + (size_t)s * b.stage_bytes;
                    const char *src = tbase + (size_t)row * row_bytes + (size_t)c0 * 512u;
                    if (b.ntiles == 1) {
                        bulk_g2s(dst, src, 4u * piece, full + s);     // 4 contiguous rows
                    } else {
#pragma unroll
                        for (int kz = 0; kz < 4; ++kz)
                            bulk_g2s(dst + kz * piece, src + kz * row_bytes, piece, full + s);
                    }
                }
                __syncwarp();
                ++k;
            }
        }
        if (!ok && lane == 0) atomicOr(p.status, BLIP_STATUS_TIMEOUT);
        // drain: every issued stage must have landed before the CTA may exit
        for (long long j = (k > S ? k - S : 0); j < k; ++j) {
            const bool got = mbar_wait(full + (int)(j % S), (unsigned)((j / S) & 1));
            if (!__all_sync(FULL, got)) {
                if (lane == 0) atomicOr(p.status, BLIP_STATUS_TIMEOUT);
                break;
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    const int cw = warp - 1;                       // chunk of the tile this warp owns
    WarpWeights &ww = wts[cw];
    long long k = 0;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int tile = (int)(it % b.ntiles);
        const int chunk = tile * b.tw + cw;
        const int nc = min(b.tw, p.nchunk - tile * b.tw);
        const bool active = cw < nc;
        const unsigned piece = (unsigned)nc * 512u;
        float acc[NW][VEC];
#pragma unroll
        for (int q = 0; q < NW; ++q)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[q][v] = 0.0f;
        int e = 0, bad = 0;
        for (int col = 0; col < 16; ++col) {
            const int s = (int)(k % S);
            const bool got = mbar_wait(full + s, (unsigned)((k / S) & 1));
            if (!__all_sync(FULL, got)) {
                if (lane == 0) atomicOr(p.status, BLIP_STATUS_TIMEOUT);
                return;
            }
            if (col == 0) {
                const ItemDesc d = desc[s];
                e = d.e;
                bad = d.bad;
                __syncwarp();
                if (!(bad & BLIP_STATUS_NONFINITE_POS)) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int pt = lane + 32 * h;
                        site_weights(p.geo, d.t[0], d.t[1], d.t[2], pt, ww.w4[pt], ww.wl[pt]);
                    }
                }
                __syncwarp();
            }
            if (active && !(bad & BLIP_STATUS_NONFINITE_POS)) {
                const unsigned char *src = stage0 + (size_t)s * b.stage_bytes + cw * 512 + lane * 16;
#pragma unroll
                for (int kz = 0; kz < 4; ++kz) {
                    const uint4 raw = *reinterpret_cast<const uint4 *>(src + kz * piece);
                    const float4 w = ww.w4[col * 4 + kz];
                    const float wl = VONLY ? 0.0f : ww.wl[col * 4 + kz];
                    float f[VEC];
                    Elt<T>::unpack(raw, f);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        acc[0][v] = fmaf(w.x, f[v], acc[0][v]);
                        if constexpr (!VONLY) {
                            acc[1][v] = fmaf(w.y, f[v], acc[1][v]);
                            acc[2][v] = fmaf(w.z, f[v], acc[2][v]);
                            acc[3][v] = fmaf(w.w, f[v], acc[3][v]);
                            acc[4][v] = fmaf(wl, f[v], acc[4][v]);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0 && !(b.stall && k == 0)) mbar_arrive(empty + s);
            ++k;
        }
        if (bad && lane == 0 && cw == 0 && tile == 0) atomicOr(p.status, bad);
        if (active) {
            if (bad & BLIP_STATUS_NONFINITE_POS) {
#pragma unroll
                for (int q = 0; q < NW; ++q)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[q][v] = __int_as_float(0x7fc00000);
            }
            store_chunk<VEC, VONLY>(p, e, chunk, lane, acc);
        }
    }
}

template <typename T, bool VONLY>
cudaError_t launch_bulk_t(const EvalParams &p, int tw, int stages, int ctas_per_sm, int sm_count,
                          int stall, cudaStream_t stream)
{
    BulkArgs b;
    b.stall = stall;
    b.tw = tw;
    b.ntiles = (p.nchunk + tw - 1) / tw;
    b.stages = stages;
    b.stage_bytes = 4 * tw * 512;
    const size_t smem = (size_t)stages * b.stage_bytes + 2 * sizeof(uint64_t) * stages
                      + sizeof(ItemDesc) * stages + sizeof(WarpWeights) * tw;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    static bool attr_set = false;   // raise this instantiation's dynamic shared-memory cap once
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(blip_eval_bulk<T, VONLY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const long long items = (long long)p.n_elec * b.ntiles;
    long long grid = (long long)sm_count * ctas_per_sm;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    blip_eval_bulk<T, VONLY><<<(unsigned)grid, 32 * (tw + 1), smem, stream>>>(p, b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bulk_elem(const EvalParams &p, int tw, int stages, int ctas_per_sm,
                             int sm_count, int stall, cudaStream_t stream)
{
    if (p.grads) return launch_bulk_t<T, false>(p, tw, stages, ctas_per_sm, sm_count, stall, stream);
    return launch_bulk_t<T, true>(p, tw, stages, ctas_per_sm, sm_count, stall, stream);
}

}  // namespace

size_t bulk_smem_bytes(int tw, int stages)
{
    return (size_t)stages * 4 * tw * 512 + 2 * sizeof(uint64_t) * stages
         + sizeof(ItemDesc) * stages + sizeof(WarpWeights) * tw;
}

cudaError_t launch_bulk(const EvalParams &p, int elem, int tw, int stages, int ctas_per_sm,
                        int sm_count, int stall, cudaStream_t stream)
{
    if (tw < 1 || tw > 8 || stages < 2 || stages > 64 || ctas_per_sm < 1) return cudaErrorInvalidValue;
    switch (elem) {
    case ELEM_F32:
        return launch_bulk_elem<float>(p, tw, stages, ctas_per_sm, sm_count, stall, stream);
    case ELEM_BF16:
        return launch_bulk_elem<__nv_bfloat16>(p, tw, stages, ctas_per_sm, sm_count, stall, stream);
    case ELEM_F16:
        return launch_bulk_elem<__half>(p, tw, stages, ctas_per_sm, sm_count, stall, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip
