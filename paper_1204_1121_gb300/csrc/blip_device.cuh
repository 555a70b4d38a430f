// Device helpers shared by the evaluation kernels: the 1-D cubic B-spline
// factors, the FP64 cell reduction, the 64 x 5 combined weights, the
// unpacking of stored elements, the packed accumulators and the output
// stores.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "blip_internal.h"
#include "../../include/blip.h"

namespace blip {
namespace dev {

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

// 16-byte read-only load that allocates in L1: used when the warps of one
// block read the same stencil rows (consecutive electrons of a sorted batch).
__device__ __forceinline__ uint4 ldg_shared_rows(const void *p)
{
    uint4 r;
    asm("ld.global.nc.L1::evict_last.v4.u32 {%0,%1,%2,%3}, [%4];"
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

// Accumulators of the five outputs (value, d/dx, d/dy, d/dz, Laplacian) of
// VEC consecutive stored elements, in packed pairs of neighbouring elements.
// Each lane of a packed FMA computes the same fma as the scalar form, so the
// results do not change; the FMA instructions per element halve.
template <int VEC>
struct AccPairs {
    float2 p[5][VEC / 2];
};

template <int VEC>
__device__ __forceinline__ void pairs_zero(AccPairs<VEC> &a)
{
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int i = 0; i < VEC / 2; ++i) a.p[k][i] = make_float2(0.0f, 0.0f);
}

// a += w_k * f for the five weights of one stencil site.
template <int VEC>
__device__ __forceinline__ void pairs_fma(AccPairs<VEC> &a, const float4 &w, float wl,
                                          const float (&f)[VEC])
{
    const float2 wk[5] = {make_float2(w.x, w.x), make_float2(w.y, w.y), make_float2(w.z, w.z),
                          make_float2(w.w, w.w), make_float2(wl, wl)};
#pragma unroll
    for (int i = 0; i < VEC / 2; ++i) {
        const float2 ff = make_float2(f[2 * i], f[2 * i + 1]);
#pragma unroll
        for (int k = 0; k < 5; ++k) a.p[k][i] = __ffma2_rn(wk[k], ff, a.p[k][i]);
    }
}

// Unpack into acc[k][v] (k = output, v = element).
template <int VEC>
__device__ __forceinline__ void pairs_out(const AccPairs<VEC> &a, float (&acc)[5][VEC])
{
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int i = 0; i < VEC / 2; ++i) {
            acc[k][2 * i] = a.p[k][i].x;
            acc[k][2 * i + 1] = a.p[k][i].y;
        }
}

// Per-warp shared-memory slice: 64 x {value, grad x, grad y, grad z} weights,
// 64 Laplacian weights, 16 stencil-column row indices.
struct WarpSlice {
    float4 w4[64];
    float wl[64];
    int colrow[16];
    float2 phase[kMaxKpoints];   // exp(2 pi i kappa_q . u) per k-point (Bloch tables)
};

// Combined weights of one electron: 64 x {value, grad x, grad y, grad z}
// and 64 Laplacian weights.
struct WarpWeights {
    float4 w4[64];
    float wl[64];
};

// FP64 reduction of position r to the base cell and offset along lattice
// direction a (Eq. 7: the 4 sites per direction around r): u = (A^{-1} r)_a,
// wrapped into [0, 1) (a tiny negative u that rounds up to 1 is the origin),
// g = n_a u, i = floor(g) mod n_a, t = g - floor(g).  Returns status bits.
__device__ __forceinline__ int wrap_axis(const Geometry &geo, int a, double rx, double ry,
                                         double rz, int &i_out, float &t_out, double *u_out = nullptr)
{
    const double *ai = geo.ainv + 3 * a;
    const double u = fma(ai[0], rx, fma(ai[1], ry, ai[2] * rz));
    if (u_out) *u_out = u;
    i_out = 0;
    t_out = 0.0f;
    if (!isfinite(u)) return BLIP_STATUS_NONFINITE_POS;
    const int bad = fabs(u) > 1099511627776.0 ? BLIP_STATUS_FAR_POS : 0;   // 2^40
    double w = u - floor(u);
    if (w >= 1.0) w = 0.0;
    const int n = geo.n[a];
    const double g = (double)n * w;
    const double fi = floor(g);
    t_out = (float)(g - fi);
    int i = (int)fi;
    if (i >= n) i -= n;
    i_out = i;
    return bad;
}

// Combined weights of stencil site pt = 16 kx + 4 ky + kz for offsets
// (t0, t1, t2): value, Cartesian gradient (sum_a J[a][c] d_a Theta) and
// Laplacian (sum_ab M_ab d_a d_b Theta), times the normalisation.
__device__ __forceinline__ void site_weights(const Geometry &geo, float t0, float t1, float t2,
                                             int pt, float4 &w4, float &wl)
{
    const int kx = pt >> 4, ky = (pt >> 2) & 3, kz = pt & 3;
    float X0, X1, X2, Y0, Y1, Y2, Z0, Z1, Z2;
    bspline_1d(t0, kx, X0, X1, X2);
    bspline_1d(t1, ky, Y0, Y1, Y2);
    bspline_1d(t2, kz, Z0, Z1, Z2);
    const float *J = geo.J, *M = geo.M;
    const float v = X0 * Y0 * Z0;
    const float gx = X1 * Y0 * Z0, gy = X0 * Y1 * Z0, gz = X0 * Y0 * Z1;
    const float wx = J[0] * gx + J[3] * gy + J[6] * gz;
    const float wy = J[1] * gx + J[4] * gy + J[7] * gz;
    const float wz = J[2] * gx + J[5] * gy + J[8] * gz;
    const float hxx = X2 * Y0 * Z0, hyy = X0 * Y2 * Z0, hzz = X0 * Y0 * Z2;
    const float hxy = X1 * Y1 * Z0, hxz = X1 * Y0 * Z1, hyz = X0 * Y1 * Z1;
    const float lap = M[0] * hxx + M[1] * hyy + M[2] * hzz
                    + 2.0f * (M[3] * hxy + M[4] * hxz + M[5] * hyz);
    const float nrm = geo.norm;
    w4 = make_float4(nrm * v, nrm * wx, nrm * wy, nrm * wz);
    wl = nrm * lap;
}

// Stored row of stencil column c = 4 kx + ky for base cell (i0, i1, i2): the
// table keeps one ghost plane below z = 0, so site z-index i2 - 1 + kz is
// stored row i2 + kz of the column.
__device__ __forceinline__ int column_row(const Geometry &geo, int i0, int i1, int i2, int c)
{
    const int n1 = geo.n[0], n2 = geo.n[1], n3 = geo.n[2];
    int ix = i0 - 1 + (c >> 2), iy = i1 - 1 + (c & 3);
    ix += ix < 0 ? n1 : 0;
    ix -= ix >= n1 ? n1 : 0;
    iy += iy < 0 ? n2 : 0;
    iy -= iy >= n2 ? n2 : 0;
    return (ix * n2 + iy) * (n3 + 3) + i2;
}

// Steps 1-2 for electron e: FP64 wrap on lanes 0-2, then weights and column
// rows into the warp's slice.  Returns the warp-uniform status bits.
// Geometry half of the per-electron setup: FP64 wrap on lanes 0-2, the 16
// stencil-column rows into the warp's slice (and the Bloch phases), then a
// __syncwarp.  Returns the warp-uniform status bits; t0..t2 receive the
// FP32 offsets for stencil_weights_warp.
// GEO: 0 = FP64 wrap here, 1 = FP64 wrap + Bloch phases, 2 = read the
// per-slot record the sort pre-pass made (its FP64 wrap already done).
// src, if given, replaces the global source: electron e's 3 coordinates
// (GEO 0, 1) or slot's record (GEO 2), e.g. a copy prefetched into shared
// memory.
template <int GEO = 0>
__device__ __forceinline__ int stencil_geometry_warp(const EvalParams &p, int e, int lane,
                                                     WarpSlice &ws, float &t0, float &t1,
                                                     float &t2, int slot = -1,
                                                     const void *src = nullptr)
{
    constexpr bool BLOCH = GEO == 1;
    if constexpr (GEO == 2) {
        // geometry already reduced in FP64 by the sort pre-pass
        const ElecGeo *rec = src ? static_cast<const ElecGeo *>(src) : p.georec + slot;
        const int4 gi = *reinterpret_cast<const int4 *>(rec);
        const float4 gt = *reinterpret_cast<const float4 *>(&rec->t[0]);
        t0 = gt.x;
        t1 = gt.y;
        t2 = gt.z;
        if (gi.w & BLIP_STATUS_NONFINITE_POS) return gi.w;
        if (lane < 16) ws.colrow[lane] = column_row(p.geo, gi.x, gi.y, gi.z, lane);
        __syncwarp();
        return gi.w;
    } else {
    int ia = 0, bad = 0;
    float ta = 0.0f;
    double ua = 0.0;
    if (lane < 3) {
        const double *r = src ? static_cast<const double *>(src) : p.pos + 3 * (size_t)e;
        bad = wrap_axis(p.geo, lane, r[0], r[1], r[2], ia, ta, &ua);
    }
    bad = __reduce_or_sync(FULL, bad);
    if constexpr (BLOCH) {
        // Bloch phases from the unwrapped fractional coordinates (FP64
        // reduction of kappa . u mod 1, then an FP32 sin/cos of 2 pi x)
        const double u0 = __shfl_sync(FULL, ua, 0), u1 = __shfl_sync(FULL, ua, 1),
                     u2 = __shfl_sync(FULL, ua, 2);
        for (int q = lane; q < p.n_k && !(bad & BLIP_STATUS_NONFINITE_POS); q += 32) {
            const double *kf = p.kfrac[q];
            const double x = fma(kf[0], u0, fma(kf[1], u1, kf[2] * u2));
            float sn, cs;
            sincospif(2.0f * (float)(x - floor(x)), &sn, &cs);
            ws.phase[q] = make_float2(cs, sn);
        }
    }
    const int i0 = __shfl_sync(FULL, ia, 0), i1 = __shfl_sync(FULL, ia, 1),
              i2 = __shfl_sync(FULL, ia, 2);
    t0 = __shfl_sync(FULL, ta, 0);
    t1 = __shfl_sync(FULL, ta, 1);
    t2 = __shfl_sync(FULL, ta, 2);
    if (bad & BLIP_STATUS_NONFINITE_POS) return bad;
    if (lane < 16) ws.colrow[lane] = column_row(p.geo, i0, i1, i2, lane);
    __syncwarp();
    return bad;
    }
}

// Weights half: the 64 x 5 combined weights into the warp's slice (two
// sites per lane), then a __syncwarp.
__device__ __forceinline__ void stencil_weights_warp(const EvalParams &p, float t0, float t1,
                                                     float t2, int lane, WarpSlice &ws)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int pt = lane + 32 * h;
        site_weights(p.geo, t0, t1, t2, pt, ws.w4[pt], ws.wl[pt]);
    }
    __syncwarp();
}

// Both halves: everything a warp needs before contracting electron e.
template <int GEO = 0>
__device__ __forceinline__ int stencil_setup_warp(const EvalParams &p, int e, int lane,
                                                  WarpSlice &ws, int slot = -1)
{
    float t0, t1, t2;
    const int bad = stencil_geometry_warp<GEO>(p, e, lane, ws, t0, t1, t2, slot);
    if (bad & BLIP_STATUS_NONFINITE_POS) return bad;
    stencil_weights_warp(p, t0, t1, t2, lane, ws);
    return bad;
}

// Scale (quantised tables) and write the five outputs of one chunk
// (32 lanes x VEC components) of electron e with streaming stores.
// Bloch factor on the (re, im) pairs of one lane's components:
// psi = ph u, grad psi = ph (grad u + i k u),
// lap psi = ph (lap u + 2 i k . grad u - |k|^2 u).
template <int VEC, bool VONLY>
__device__ __forceinline__ void apply_bloch(const EvalParams &p, int l0, const float2 *phase,
                                            float (&acc)[VONLY ? 1 : 5][VEC])
{
#pragma unroll
    for (int v = 0; v < VEC; v += 2) {
        // the k-point of complex orbital lc: the last q with koff[q] <= lc
        const int lc = (l0 + v) >> 1;
        int q = 0, hi = p.n_k;
        while (hi - q > 1) {
            const int mid = (q + hi) >> 1;
            if (p.koff[mid] <= lc) q = mid;
            else hi = mid;
        }
        const float2 ph = phase[q];
        const float ur = acc[0][v], ui = acc[0][v + 1];
        acc[0][v] = ph.x * ur - ph.y * ui;
        acc[0][v + 1] = ph.x * ui + ph.y * ur;
        if constexpr (!VONLY) {
            const float k0 = p.kcart[q][0], k1 = p.kcart[q][1], k2 = p.kcart[q][2];
            const float kk[3] = {k0, k1, k2};
            float kgr = 0.0f, kgi = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float gr = acc[1 + c][v], gi = acc[1 + c][v + 1];
                kgr = fmaf(kk[c], gr, kgr);
                kgi = fmaf(kk[c], gi, kgi);
                const float tr = gr - kk[c] * ui, ti = gi + kk[c] * ur;
                acc[1 + c][v] = ph.x * tr - ph.y * ti;
                acc[1 + c][v + 1] = ph.x * ti + ph.y * tr;
            }
            const float ksq = k0 * k0 + k1 * k1 + k2 * k2;
            const float tr = acc[4][v] - 2.0f * kgi - ksq * ur;
            const float ti = acc[4][v + 1] + 2.0f * kgr - ksq * ui;
            acc[4][v] = ph.x * tr - ph.y * ti;
            acc[4][v + 1] = ph.x * ti + ph.y * tr;
        }
    }
}

template <int VEC, bool VONLY, bool BLOCH = false>
__device__ __forceinline__ void store_chunk(const EvalParams &p, int e, int chunk, int lane,
                                            float (&acc)[VONLY ? 1 : 5][VEC],
                                            const float2 *phase = nullptr)
{
    constexpr int NW = VONLY ? 1 : 5;
    const size_t L = (size_t)p.Lreal;
    const int l0 = chunk * 32 * VEC + lane * VEC;
    if (l0 >= p.Lreal) return;
    if (p.scales) {
#pragma unroll
        for (int v = 0; v < VEC; v += 4) {
            const float4 s = *reinterpret_cast<const float4 *>(p.scales + l0 + v);
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                acc[k][v] *= s.x; acc[k][v + 1] *= s.y;
                acc[k][v + 2] *= s.z; acc[k][v + 3] *= s.w;
            }
        }
    }
    if constexpr (BLOCH) apply_bloch<VEC, VONLY>(p, l0, phase, acc);
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
                       make_float4(acc[k][v], acc[k][v + 1], acc[k][v + 2], acc[k][v + 3]));
    } else {
        const int nv = min(VEC, p.Lreal - l0);
#pragma unroll
        for (int k = 0; k < NW; ++k)
#pragma unroll
            for (int v = 0; v < VEC; ++v)
                if (v < nv) __stcs(dst[k] + v, acc[k][v]);
    }
}

// Walker offsets check (any thread of the grid): offsets[0] = 0, monotone,
// offsets[n_walkers] = n_elec.
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


}  // namespace dev
}  // namespace blip
