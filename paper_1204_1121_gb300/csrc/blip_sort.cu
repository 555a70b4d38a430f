// Spatial sort pre-pass: order the electrons of a batch by the grid cell that
// holds them, so that the warps running at the same time read overlapping
// stencil rows and the L2 cache serves the repeats.  This is the batching
// step that turns the quasi-simultaneous update's N independent evaluations
// (Sec. IV.A, Eq. 11.12.23.1) into cache-friendly work; the paper itself
// evaluates in input order.
//
// The order is brick-major (sort_cell_key): the (a_1, a_2) plane is cut into
// 8 x 8 bricks of whole z-columns, grouped 4 x 4 into super-bricks; super-
// bricks and the bricks inside them in row-major order, and inside a brick
// the cells in row-major order with z fastest (the table's own row order).
// A window of consecutively evaluated electrons then covers a compact 3-D
// region, so the rows its stencils share along a_1 and a_2 are still in L2
// when reused; with a plain row-major cell order the a_1 neighbours come one
// whole (a_2, a_3) plane later, and with row-major bricks alone a whole row
// of bricks later.
//
// Counting sort over these cell keys (plus one bucket for positions without
// a cell), in four kernels:
//   1. key of every electron (FP64 wrap, the same reduction as the
//      evaluation) and a histogram of keys (atomicAdd),
//   2-3. exclusive scan of the histogram (tile scans, then a scan of the tile
//      totals and their addition),
//   4. scatter: perm[atomicAdd(cursor[key], 1)] = e.
// The order inside one cell is not deterministic, but every electron's result
// is computed independently, so the outputs are.
#include "blip_internal.h"
#include "../../include/blip.h"

namespace blip {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void sort_keys_kernel(Geometry geo, const double *__restrict__ pos, int n_elec,
                                 int *__restrict__ keys, int *__restrict__ hist, int P,
                                 ElecGeo *__restrict__ rec)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_elec; e += gridDim.x * blockDim.x) {
        const double rx = pos[3 * (size_t)e], ry = pos[3 * (size_t)e + 1],
                     rz = pos[3 * (size_t)e + 2];
        int idx[3];
        float tt[3];
        int badbits = 0;
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // the same FP64 reduction as the evaluation kernels' wrap
            const double u = fma(geo.ainv[3 * a], rx, fma(geo.ainv[3 * a + 1], ry,
                                                          geo.ainv[3 * a + 2] * rz));
            tt[a] = 0.0f;
            if (!isfinite(u)) { ok = false; idx[a] = 0; continue; }
            if (fabs(u) > 1099511627776.0) badbits |= BLIP_STATUS_FAR_POS;   // 2^40
            double w = u - floor(u);
            if (w >= 1.0) w = 0.0;
            const double g = (double)geo.n[a] * w;
            const double fi = floor(g);
            tt[a] = (float)(g - fi);
            int i = (int)fi;
            if (i >= geo.n[a]) i -= geo.n[a];
            idx[a] = i;
        }
        if (!ok) badbits |= BLIP_STATUS_NONFINITE_POS;
        if (rec) {
            ElecGeo r;
            r.i[0] = idx[0]; r.i[1] = idx[1]; r.i[2] = idx[2];
            r.bad = badbits;
            r.t[0] = tt[0]; r.t[1] = tt[1]; r.t[2] = tt[2];
            r.pad = 0.0f;
            rec[e] = r;
        }
        const int key = ok ? sort_cell_key(geo, idx[0], idx[1], idx[2]) : P;
        keys[e] = key;
        atomicAdd(hist + key, 1);
    }
}

// Exclusive scan of one 4096-element tile per block; tile totals to sums.
__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles_kernel(int *__restrict__ data, int n,
                                                                 int *__restrict__ sums)
{
    __shared__ int warp_tot[SCAN_THREADS / 32];
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? data[base + i] : 0;
        s += v[i];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = warp_tot[lane];
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        warp_tot[lane] = ti - t;               // exclusive warp offsets
        if (lane == 31) sums[blockIdx.x] = ti;  // tile total
    }
    __syncthreads();
    int run = warp_tot[wid] + incl - s;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
}

__global__ void add_tile_offsets_kernel(int *__restrict__ data, int n, const int *__restrict__ offs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) data[i] += offs[i / SCAN_TILE];
}

__global__ void sort_scatter_kernel(const int *__restrict__ keys, int n_elec,
                                    int *__restrict__ cursor, int *__restrict__ perm,
                                    const ElecGeo *__restrict__ rec,
                                    ElecGeo *__restrict__ rec_sorted)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_elec; e += gridDim.x * blockDim.x) {
        const int slot = atomicAdd(cursor + keys[e], 1);
        perm[slot] = e;
        if (rec_sorted) rec_sorted[slot] = rec[e];
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Cell keys (sort_cell_key): whole 32 x 32 super-bricks of z-columns, so the
// key range covers the grid rounded up to multiples of 32 along a_1 and a_2.
long long sort_buckets(const Geometry &geo) { return sort_key_count(geo); }

}  // namespace

size_t sort_scratch_bytes(int n_elec, const Geometry &geo)
{
    const long long nb = sort_buckets(geo) + 1;
    const long long tiles = (nb + SCAN_TILE - 1) / SCAN_TILE;
    return align256(sizeof(int) * (size_t)nb) + 2 * align256(sizeof(int) * (size_t)n_elec)
         + 2 * align256(sizeof(int) * (size_t)(tiles + 1));
}

// Views into a sorted scratch: keys[e] of every electron and, after the
// scatter, cell_end[k] = one past the last slot of key k (so key k occupies
// slots [k ? cell_end[k - 1] : 0, cell_end[k])).
void sort_views(const Geometry &geo, int n_elec, void *scratch, const int **keys,
                const int **cell_end)
{
    const long long nb = sort_buckets(geo) + 1;
    char *c = static_cast<char *>(scratch);
    *cell_end = reinterpret_cast<const int *>(c);
    *keys = reinterpret_cast<const int *>(c + align256(sizeof(int) * (size_t)nb));
    (void)n_elec;
}

// Scratch layout: hist[P + 1] | keys[n_elec] | perm[n_elec] | sums | sums2.
cudaError_t launch_sort(const Geometry &geo, const double *pos, int n_elec, void *scratch,
                        int **perm_out, cudaStream_t stream, ElecGeo *rec_by_e,
                        ElecGeo *rec_by_slot)
{
    if ((rec_by_e == nullptr) != (rec_by_slot == nullptr)) return cudaErrorInvalidValue;
    const int P = (int)sort_buckets(geo);
    const int nb = P + 1;
    const int tiles = (nb + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles > SCAN_TILE) return cudaErrorInvalidValue;   // > 16.7M cells
    char *c = static_cast<char *>(scratch);
    int *hist = reinterpret_cast<int *>(c);
    c += align256(sizeof(int) * (size_t)nb);
    int *keys = reinterpret_cast<int *>(c);
    c += align256(sizeof(int) * (size_t)n_elec);
    int *perm = reinterpret_cast<int *>(c);
    c += align256(sizeof(int) * (size_t)n_elec);
    int *sums = reinterpret_cast<int *>(c);
    c += align256(sizeof(int) * (size_t)(tiles + 1));
    int *sums2 = reinterpret_cast<int *>(c);

    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * (size_t)nb, stream);
    if (e != cudaSuccess) return e;
    const int eb = (n_elec + 255) / 256;
    sort_keys_kernel<<<eb < 1 ? 1 : (eb > 65535 * 8 ? 65535 * 8 : eb), 256, 0, stream>>>(
        geo, pos, n_elec, keys, hist, P, rec_by_e);
    scan_tiles_kernel<<<tiles, SCAN_THREADS, 0, stream>>>(hist, nb, sums);
    scan_tiles_kernel<<<1, SCAN_THREADS, 0, stream>>>(sums, tiles, sums2);
    add_tile_offsets_kernel<<<(nb + 255) / 256, 256, 0, stream>>>(hist, nb, sums);
    sort_scatter_kernel<<<eb < 1 ? 1 : (eb > 65535 * 8 ? 65535 * 8 : eb), 256, 0, stream>>>(
        keys, n_elec, hist, perm, rec_by_e, rec_by_slot);
    *perm_out = perm;
    return cudaGetLastError();
}

}  // namespace blip
