// Evaluation kernels: values, gradients and Laplacians of all orbitals at a
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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "blip_internal.h"
#include "../../include/blip.h"

namespace blip {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// 1-D cubic B-spline factor (value, d/dg, d2/dg2) for stencil site k = 0..3
// of an electron at offset t in [0, 1) from its base site: the site sits at
// grid distance x = t + 1 - k.  Polynomial forms of the piecewise definition
// (Eq. 11.12.24.2 with phi the cubic B-spline), s = 1 - t.
__device__ __forceinline__ void bspline_1d(float t, int k, float &b, float &d1, float &d2)
{
    const float s = 1.0f - t;
    if (k == 0) {          // x = t + 1 in [1, 2)
        b = s * s * s * (1.0f / 6.0f);
        d1 = -0.5f * s * s;
        d2 = s;
    } else if (k == 1) {   // x = t in [0, 1)
        b = fmaf(0.5f * t - 1.0f, t * t, 2.0f / 3.0f);
        d1 = (1.5f * t - 2.0f) * t;
        d2 = fmaf(3.0f, t, -2.0f);
    } else if (k == 2) {   // x = t - 1 in [-1, 0)
        b = fmaf(0.5f * s - 1.0f, s * s, 2.0f / 3.0f);
        d1 = -(1.5f * s - 2.0f) * s;
        d2 = fmaf(3.0f, s, -2.0f);
    } else {               // x = t - 2 in [-2, -1)
        b = t * t * t * (1.0f / 6.0f);
        d1 = 0.5f * t * t;
        d2 = t;
    }
}

// 16-byte read-only load that bypasses L1 and asks L2 for 256-byte sectors
// (the 4 rows of a stencil column are long contiguous runs).
__device__ __forceinline__ uint4 ldg_stream(const void *p)
{
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}

template <typename T> struct Elt;
template <> struct Elt<float> {
    static constexpr int VEC = 4;
    static __device__ __forceinline__ void unpack(const uint4 &r, float *f)
    {
        f[0] = __uint_as_float(r.x); f[1] = __uint_as_float(r.y);
        f[2] = __uint_as_float(r.z); f[3] = __uint_as_float(r.w);
    }
};
template <> struct Elt<__nv_bfloat16> {
    static constexpr int VEC = 8;
    static __device__ __forceinline__ void unpack(const uint4 &r, float *f)
    {
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            f[2 * i] = __uint_as_float(w[i] << 16);
            f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};
template <> struct Elt<__half> {
    static constexpr int VEC = 8;
    static __device__ __forceinline__ void unpack(const uint4 &r, float *f)
    {
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h = *reinterpret_cast<const __half2 *>(&w[i]);
            float2 v = __half22float2(h);
            f[2 * i] = v.x;
            f[2 * i + 1] = v.y;
        }
    }
};

// Per-warp shared-memory slice: 64 x {value, grad x, grad y, grad z} weights,
// 64 Laplacian weights, 16 stencil-column row indices.
struct WarpSlice {
    float4 w4[64];
    float wl[64];
    int colrow[16];
};

// Steps 1-2 for electron e: FP64 wrap on lanes 0-2, then weights and column
// rows into the warp's slice.  Returns the warp-uniform status bits.
__device__ __forceinline__ int stencil_setup(const EvalParams &p, int e, int lane, WarpSlice &ws)
{
    int ia = 0, bad = 0;
    float ta = 0.0f;
    if (lane < 3) {
        const double *r = p.pos + 3 * (size_t)e;
        const double rx = r[0], ry = r[1], rz = r[2];
        const double *ai = p.geo.ainv + 3 * lane;
        const double u = fma(ai[0], rx, fma(ai[1], ry, ai[2] * rz));
        if (!isfinite(u)) {
            bad = BLIP_STATUS_NONFINITE_POS;
        } else {
            if (fabs(u) > 1099511627776.0) bad = BLIP_STATUS_FAR_POS;   // 2^40
            double w = u - floor(u);
            if (w >= 1.0) w = 0.0;            // tiny negative u rounds up to 1: the origin
            const int n = p.geo.n[lane];
            const double g = (double)n * w;
            const double fi = floor(g);
            ta = (float)(g - fi);
            ia = (int)fi;
            if (ia >= n) ia -= n;
        }
    }
    bad = __reduce_or_sync(FULL, bad);
    const int i0 = __shfl_sync(FULL, ia, 0), i1 = __shfl_sync(FULL, ia, 1),
              i2 = __shfl_sync(FULL, ia, 2);
    const float t0 = __shfl_sync(FULL, ta, 0), t1 = __shfl_sync(FULL, ta, 1),
                t2 = __shfl_sync(FULL, ta, 2);
    if (bad & BLIP_STATUS_NONFINITE_POS) return bad;

    const float *J = p.geo.J, *M = p.geo.M;
    const float nrm = p.geo.norm;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int pt = lane + 32 * h;
        const int kx = pt >> 4, ky = (pt >> 2) & 3, kz = pt & 3;
        float X0, X1, X2, Y0, Y1, Y2, Z0, Z1, Z2;
        bspline_1d(t0, kx, X0, X1, X2);
        bspline_1d(t1, ky, Y0, Y1, Y2);
        bspline_1d(t2, kz, Z0, Z1, Z2);
        const float v = X0 * Y0 * Z0;
        const float gx = X1 * Y0 * Z0, gy = X0 * Y1 * Z0, gz = X0 * Y0 * Z1;
        const float wx = J[0] * gx + J[3] * gy + J[6] * gz;   // sum_a J[a][c] dg_a
        const float wy = J[1] * gx + J[4] * gy + J[7] * gz;
        const float wz = J[2] * gx + J[5] * gy + J[8] * gz;
        const float hxx = X2 * Y0 * Z0, hyy = X0 * Y2 * Z0, hzz = X0 * Y0 * Z2;
        const float hxy = X1 * Y1 * Z0, hxz = X1 * Y0 * Z1, hyz = X0 * Y1 * Z1;
        const float lap = M[0] * hxx + M[1] * hyy + M[2] * hzz
                        + 2.0f * (M[3] * hxy + M[4] * hxz + M[5] * hyz);
        ws.w4[pt] = make_float4(nrm * v, nrm * wx, nrm * wy, nrm * wz);
        ws.wl[pt] = nrm * lap;
    }
    if (lane < 16) {
        const int n1 = p.geo.n[0], n2 = p.geo.n[1], n3 = p.geo.n[2];
        int ix = i0 - 1 + (lane >> 2), iy = i1 - 1 + (lane & 3);
        ix += ix < 0 ? n1 : 0;  ix -= ix >= n1 ? n1 : 0;
        iy += iy < 0 ? n2 : 0;  iy -= iy >= n2 ? n2 : 0;
        // stored z-row of site i2 - 1 + kz is i2 + kz (one ghost plane below)
        ws.colrow[lane] = (ix * n2 + iy) * (n3 + 3) + i2;
    }
    __syncwarp();
    return bad;
}

template <int CPW, int VEC, bool VONLY>
__device__ __forceinline__ void store_outputs(const EvalParams &p, int e, int grp, int lane,
                                              float (&acc)[CPW][VONLY ? 1 : 5][VEC])
{
    constexpr int NW = VONLY ? 1 : 5;
    const size_t L = (size_t)p.Lreal;
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
        const int chunk = grp * CPW + c;
        if (chunk >= p.nchunk) break;                    // warp-uniform
        const int l0 = chunk * 32 * VEC + lane * VEC;
        if (l0 >= p.Lreal) continue;
        if (p.scales) {
#pragma unroll
            for (int v = 0; v < VEC; v += 4) {
                const float4 s = *reinterpret_cast<const float4 *>(p.scales + l0 + v);
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    acc[c][k][v] *= s.x; acc[c][k][v + 1] *= s.y;
                    acc[c][k][v + 2] *= s.z; acc[c][k][v + 3] *= s.w;
                }
            }
        }
        float *dst[5];
        dst[0] = p.values + (size_t)e * L + l0;
        if constexpr (!VONLY) {
            dst[1] = p.grads + (size_t)e * 3 * L + l0;
            dst[2] = dst[1] + L;
            dst[3] = dst[1] + 2 * L;
            dst[4] = p.laps + (size_t)e * L + l0;
        }
        if (p.vec_out && l0 + VEC <= p.Lreal) {
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; v += 4)
                    __stcs(reinterpret_cast<float4 *>(dst[k] + v),
                           make_float4(acc[c][k][v], acc[c][k][v + 1], acc[c][k][v + 2],
                                       acc[c][k][v + 3]));
        } else {
            const int nv = min(VEC, p.Lreal - l0);
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                    if (v < nv) __stcs(dst[k] + v, acc[c][k][v]);
        }
    }
}

__device__ __forceinline__ void check_offsets(const EvalParams &p)
{
    if (!p.offsets) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= p.n_walkers;
         i += stride) {
        const int o = p.offsets[i];
        bool ok = (i == 0) ? (o == 0) : (o >= p.offsets[i - 1]);
        ok = ok && (i == p.n_walkers ? o == p.n_elec : o <= p.n_elec);
        if (!ok) atomicOr(p.status, BLIP_STATUS_BAD_OFFSETS);
    }
}

// Register-gather kernel: each lane loads its 16-byte slices of the 64 rows
// straight into registers (4 columns = 16 rows in flight per batch for one
// chunk, fewer for more chunks).
template <typename T, int CPW, bool VONLY>
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

    for (long long item = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); item < p.items;
         item += nwarps) {
        const int slot = (int)(item / p.groups);
        const int grp = (int)(item - (long long)slot * p.groups);
        const int e = p.perm ? p.perm[slot] : slot;

        float acc[CPW][NW][VEC];
#pragma unroll
        for (int c = 0; c < CPW; ++c)
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[c][k][v] = 0.0f;

        __syncwarp();                      // previous item's readers are done with the slice
        const int bad = stencil_setup(p, e, lane, ws);
        if (bad && lane == 0) atomicOr(p.status, bad);
        if (bad & BLIP_STATUS_NONFINITE_POS) {
#pragma unroll
            for (int c = 0; c < CPW; ++c)
#pragma unroll
                for (int k = 0; k < NW; ++k)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[c][k][v] = __int_as_float(0x7fc00000);
            store_outputs<CPW, VEC, VONLY>(p, e, grp, lane, acc);
            continue;
        }

        size_t coff[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
            const int chunk = min(grp * CPW + c, p.nchunk - 1);   // clamp: in-bounds duplicate
            coff[c] = ((size_t)chunk * 32 * VEC + (size_t)lane * VEC) * sizeof(T);
        }

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
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            acc[c][0][v] = fmaf(w.x, f[v], acc[c][0][v]);
                            if constexpr (!VONLY) {
                                acc[c][1][v] = fmaf(w.y, f[v], acc[c][1][v]);
                                acc[c][2][v] = fmaf(w.z, f[v], acc[c][2][v]);
                                acc[c][3][v] = fmaf(w.w, f[v], acc[c][3][v]);
                                acc[c][4][v] = fmaf(wl, f[v], acc[c][4][v]);
                            }
                        }
                    }
                }
        }
        store_outputs<CPW, VEC, VONLY>(p, e, grp, lane, acc);
    }
}

template <typename T, int CPW, bool VONLY>
cudaError_t launch_register_t(const EvalParams &p, int warps, cudaStream_t stream)
{
    const size_t smem = sizeof(WarpSlice) * (size_t)warps;
    long long blocks = (p.items + warps - 1) / warps;
    if (blocks < 1) blocks = 1;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    blip_eval_register<T, CPW, VONLY><<<(unsigned)blocks, 32 * warps, smem, stream>>>(p);
    return cudaGetLastError();
}

template <typename T, bool VONLY>
cudaError_t launch_register_c(const EvalParams &p, int chunks, int warps, cudaStream_t stream)
{
    switch (chunks) {
    case 1: return launch_register_t<T, 1, VONLY>(p, warps, stream);
    case 2: return launch_register_t<T, 2, VONLY>(p, warps, stream);
    case 3: return launch_register_t<T, 3, VONLY>(p, warps, stream);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_register(const EvalParams &p, int chunks, int warps, cudaStream_t stream)
{
    if (p.grads) return launch_register_c<T, false>(p, chunks, warps, stream);
    return launch_register_c<T, true>(p, chunks, warps, stream);
}

}  // namespace

cudaError_t launch_eval(const EvalParams &p, int elem, int variant, int chunks, int warps,
                        cudaStream_t stream)
{
    if (warps < 1 || warps > 16) return cudaErrorInvalidValue;
    (void)variant;
    switch (elem) {
    case ELEM_F32: return launch_register<float>(p, chunks, warps, stream);
    case ELEM_BF16: return launch_register<__nv_bfloat16>(p, chunks, warps, stream);
    case ELEM_F16: return launch_register<__half>(p, chunks, warps, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip
