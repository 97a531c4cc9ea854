// es_device.cuh -- small device helpers shared by the libes kernels.
#pragma once

#include <cuda_fp16.h>

#include "es_internal.cuh"

namespace es {

__device__ __forceinline__ int gdim(const Grid& g, int a) { return a == 0 ? g.nx : (a == 1 ? g.ny : g.nz); }

__device__ __forceinline__ long long lin(const Grid& g, int x, int y, int z) {
    return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
}

// Neighbour coordinate along one axis; returns false when the step leaves
// the domain through a non-periodic face.
__device__ __forceinline__ bool step_axis(int v, int d, int n, int per, int& out) {
    int p = v + d;
    if (p < 0 || p >= n) {
        if (!per) return false;
        p = p < 0 ? p + n : p - n;
    }
    out = p;
    return true;
}

__device__ __forceinline__ bool neighbour(const Grid& g, int x, int y, int z, int dx, int dy, int dz,
                                          long long& out) {
    int a, b, c;
    if (!step_axis(x, dx, g.nx, g.per[0], a)) return false;
    if (!step_axis(y, dy, g.ny, g.per[1], b)) return false;
    if (!step_axis(z, dz, g.nz, g.per[2], c)) return false;
    out = lin(g, a, b, c);
    return true;
}

// Minimum-image displacement of a cell centre (cell + 1/2) from X.
__device__ __forceinline__ double cell_disp(const Grid& g, int axis, int cell, double X) {
    double d = __dsub_rn((double)cell + 0.5, X);
    if (g.per[axis]) {
        double L = (double)gdim(g, axis);
        if (d > 0.5 * L) d = __dsub_rn(d, L);
        if (d < -0.5 * L) d = __dadd_rn(d, L);
    }
    return d;
}

// Cell-centre-in-sphere test of the moving obstacle mapping (Sec. 4.2), with
// explicit round-to-nearest operations: no FMA contraction, so the decision
// is the one an IEEE FP64 evaluation of (dx^2 + dy^2) + dz^2 <= R^2 takes.
__device__ __forceinline__ bool cell_inside(const Grid& g, const DParticle& p, int x, int y, int z) {
    double dx = cell_disp(g, 0, x, p.x[0]);
    double dy = cell_disp(g, 1, y, p.x[1]);
    double dz = cell_disp(g, 2, z, p.x[2]);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 <= __dmul_rn(p.R, p.R);
}

// FP32 distances from a sphere centre to the cells of a box [blo, bhi], for deciding
// cheaply which cells need work: the centre relative to the box origin is
// formed once in FP64 and rounded to float, so the FP32 squared distance of
// a cell (local index i, j, k) is within ~1e-6 relative of the FP64 one.
// ok is false where a periodic axis is too short for the unwrapped distance
// to be the minimum image everywhere in the box (callers then take the slow
// path for every cell).
struct BallF {
    float c[3], r2, margin;
    bool ok;
    __device__ void init(const Grid& g, const double* X, double R, const int* blo, const int* bhi) {
        ok = true;
        for (int a = 0; a < 3; a++) {
            c[a] = (float)(X[a] - ((double)blo[a] + 0.5));
            if (g.per[a]) {
                const double half = 0.5 * (double)gdim(g, a);
                const double lo = (double)blo[a] + 0.5 - X[a], hi = (double)bhi[a] + 0.5 - X[a];
                if (!(lo > -half + 1.0 && hi < half - 1.0)) ok = false;
            }
        }
        r2 = (float)(R * R);
        margin = 1e-5f * (r2 + 100.0f);  // far above the FP32 rounding of d^2
    }
    __device__ float d2(int i, int j, int k) const {
        const float dx = (float)i - c[0], dy = (float)j - c[1], dz = (float)k - c[2];
        return dx * dx + dy * dy + dz * dz;
    }
};

// The owner field over a box [lo - 1, hi + 1] (the box and a one-cell
// halo) in shared memory, x fastest; cells beyond a non-periodic face read
// kOwnerOutside.  Per-sphere kernels read a cell's D3Q19 neighbours from it
// with fixed offsets instead of wrapping indices per neighbour.
constexpr int kOwnerOutside = -0x7fffffff;
constexpr int kOwnerTileMax = 8192;  // ints of shared memory per block

struct OwnerTile {
    int n[3];  // box extents (the tile is (n + 2)^3)
    __device__ int tx() const { return n[0] + 2; }
    __device__ int txy() const { return (n[0] + 2) * (n[1] + 2); }
    __device__ bool fits(int max_ints = kOwnerTileMax) const { return (n[0] + 2) * (n[1] + 2) * (n[2] + 2) <= max_ints; }
    // tile index of the box cell with local index (i, j, k)
    __device__ int at(int i, int j, int k) const { return (i + 1) + tx() * (j + 1) + txy() * (k + 1); }
    // offset of the D3Q19 neighbour in direction q
    __device__ int step(int q) const { return cx(q) + tx() * cy(q) + txy() * cz(q); }
};

// Local indices (i, j, k) of the cells t, t + step, t + 2 step, ... of a box
// of extents sx x sy x ..., x fastest, advanced without integer division.
struct BoxWalk {
    int i, j, k, si, sj, sk, sx, sy;
    __device__ __forceinline__ void start(int t0, int step, int sx_, int sy_) {
        sx = sx_;
        sy = sy_;
        i = t0 % sx;
        j = (t0 / sx) % sy;
        k = t0 / (sx * sy);
        si = step % sx;
        sj = (step / sx) % sy;
        sk = step / (sx * sy);
    }
    __device__ __forceinline__ void next() {
        i += si;
        j += sj;
        k += sk;
        if (i >= sx) {
            i -= sx;
            j++;
        }
        if (j >= sy) {
            j -= sy;
            k++;
        }
    }
};

// v in [-n, 2n) into [0, n) (a box never spans more than one period).
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ void load_owner_tile(const Grid& g, const int32_t* __restrict__ owner, const int* lo,
                                                const OwnerTile& T, int* tile) {
    const int sx = T.n[0] + 2, sy = T.n[1] + 2, n = sx * sy * (T.n[2] + 2);
    const int dim[3] = {g.nx, g.ny, g.nz};
    BoxWalk w;
    w.start(threadIdx.x, blockDim.x, sx, sy);
    for (int t = threadIdx.x; t < n; t += blockDim.x, w.next()) {
        int v[3] = {lo[0] - 1 + w.i, lo[1] - 1 + w.j, lo[2] - 1 + w.k};
        bool out = false;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (v[a] < 0 || v[a] >= dim[a]) {
                if (!g.per[a])
                    out = true;
                else
                    v[a] = wrap1(v[a], dim[a]);
            }
        }
        tile[t] = out ? kOwnerOutside : owner[lin(g, v[0], v[1], v[2])];
    }
}

// Surface velocity u_s = V + Omega x (x_s - X) at the centre of a cell.
__device__ __forceinline__ void surface_velocity(const Grid& g, const double* X, const double* V,
                                                 const double* W, int x, int y, int z, double u[3]) {
    double r0 = cell_disp(g, 0, x, X[0]);
    double r1 = cell_disp(g, 1, y, X[1]);
    double r2 = cell_disp(g, 2, z, X[2]);
    u[0] = V[0] + (W[1] * r2 - W[2] * r1);
    u[1] = V[1] + (W[2] * r0 - W[0] * r2);
    u[2] = V[2] + (W[0] * r1 - W[1] * r0);
}

// Cell range along one axis that can hold cells within R (+ ext) of X.
// A range of n or more cells becomes the whole axis (no cell twice);
// non-periodic axes are clamped to the domain.
__device__ __forceinline__ void axis_range(const Grid& g, int a, double lo_x, double hi_x, double R,
                                           int ext, int& lo, int& hi) {
    int n = gdim(g, a);
    lo = (int)floor(lo_x - R - 0.5) - ext;
    hi = (int)ceil(hi_x + R - 0.5) + ext;
    if (hi - lo + 1 >= n) {
        lo = 0;
        hi = n - 1;
    }
    if (!g.per[a]) {
        lo = lo < 0 ? 0 : lo;
        hi = hi > n - 1 ? n - 1 : hi;
    }
}

__device__ __forceinline__ int wrap_coord(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Block-wide sum of a double in a fixed order (warp shuffles, then warp 0).
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // valid in thread 0
}

// ---- PDF storage forms ----
// What one stored population holds, and the arithmetic type C of the
// stream-collide that reads it:
//   double: f_q (FP64 form, C = double);
//   float:  f_q - w_q (MIXED32, C = float): the deviation from the rest
//           state keeps FP32 resolution for the small departures from w_q;
//   __half: 2^12 (f_q - w_q) / w_q (MIXED16, C = float): the deviation
//           relative to its weight, so that all 19 streams use FP16 alike,
//           scaled by 2^12 because FP16 is normal only from 6.1e-5 on while
//           the relative deviations of slow flows are 1e-6 .. 1e-3 (scaled,
//           they stay normal down to 1.5e-8; the largest one kept is 16).
// ld / st convert between a stored value and the collide's working value
// (f_q for double, f_q - w_q otherwise); to_f / from_f give f_q in double.
template <class S>
struct Store;

template <>
struct Store<double> {
    using C = double;
    static constexpr bool shifted = false;
    __device__ static double ld(int, double s) { return s; }
    __device__ static double st(int, double v) { return v; }
    __device__ static double rest(int q) { return wq(q); }
    __device__ static double to_f(int, double s) { return s; }
    __device__ static double from_f(int, double f) { return f; }
    __device__ static double from_dev(int q, double dev) { return wq(q) + dev; }
};

template <>
struct Store<float> {
    using C = float;
    static constexpr bool shifted = true;
    __device__ static float ld(int, float s) { return s; }
    __device__ static float st(int, float v) { return v; }
    __device__ static float rest(int) { return 0.0f; }
    __device__ static double to_f(int q, float s) { return (double)s + wq(q); }
    __device__ static float from_f(int q, double f) { return (float)(f - wq(q)); }
    __device__ static float from_dev(int, double dev) { return (float)dev; }
};

constexpr double kHalfScale = 4096.0;

template <>
struct Store<__half> {
    using C = float;
    static constexpr bool shifted = true;
    __device__ static float ld(int q, __half s) { return __half2float(s) * (float)(wq(q) / kHalfScale); }
    __device__ static __half st(int q, float v) { return __float2half_rn(v * (float)(kHalfScale / wq(q))); }
    __device__ static __half rest(int) { return __float2half_rn(0.0f); }
    __device__ static double to_f(int q, __half s) { return wq(q) + (double)__half2float(s) * (wq(q) / kHalfScale); }
    __device__ static __half from_f(int q, double f) {
        return __float2half_rn((float)((f - wq(q)) * (kHalfScale / wq(q))));
    }
    __device__ static __half from_dev(int q, double dev) { return __float2half_rn((float)(dev * (kHalfScale / wq(q)))); }
};

// ---- float-float ("double-single") arithmetic ----
// A value is held as the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significant bits.  The MIXED32 form keeps psi
// and the outer residual this way: GB300 runs FP64 arithmetic and FP64
// conversions at 1/64 of the FP32 rate, while these operations are a handful
// of FP32 additions and FMAs.  The error-free transformations are Knuth's
// TwoSum, Dekker's FastTwoSum and the FMA form of TwoProd (Muller et al.,
// Handbook of Floating-Point Arithmetic, 2nd ed., Sec. 4.3 and 4.4); the
// explicit _rn intrinsics keep the compiler from contracting or reassociating
// them.
struct ff {
    float hi, lo;
};

// s + e == a + b exactly, s = fl(a + b)
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// as two_sum, valid when |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// float-float + float-float (the accurate two-TwoSum form)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

// float-float + float
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    const ff s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// float-float * float-float (lo * lo dropped, below 2^-48 relative)
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// Sum of terms kept as a float head plus a float tail of rounding errors
// and low parts; cheaper than a chain of ff_add when terms are only added.
struct ff_acc {
    float s, t;
    __device__ __forceinline__ void add(float hi, float lo) {
        const ff r = two_sum(s, hi);
        s = r.hi;
        t = __fadd_rn(t, __fadd_rn(r.lo, lo));
    }
    __device__ __forceinline__ ff value() const { return two_sum(s, t); }
};

// The potential at an interior fluid cell (c) and at its 18 D3Q19
// neighbours, named by their offsets (xpym: x + 1, y - 1, ...).
struct Psi19 {
    float c, xp, xm, yp, ym, zp, zm;
    float xpyp, xmym, xpym, xmyp, xpzp, xmzm, xpzm, xmzp, ypzp, ymzm, ypzm, ymzp;
};

// Electric body force of the reduced forms at an interior fluid cell (Sec.
// 5.6): the isotropic D3Q19 gradient (1/c_s^2) sum_q w_q psi(x + e_q) e_q
// (Eq. ElPotGradComp) taken pairwise, 3 w_q (psi(x + e_q) - psi(x - e_q)),
// the charge density rho_e = -kappa^2 eps psi (Eq. ChrgDensDHA; k2e =
// kappa^2 eps) and f_b = rho_e (E_ext - grad psi).  Every operation is
// rounded on its own (no FMA contraction), so the stream-collide that
// evaluates it on the fly and the kernel that stores the field give the
// same bits.
__device__ __forceinline__ void body_force_iso(const Psi19& p, float Ex, float Ey, float Ez, float k2e, float& f0,
                                               float& f1, float& f2) {
    const float a = (float)(3.0 / 18.0), b = (float)(3.0 / 36.0);
    float g0 = __fmul_rn(a, __fsub_rn(p.xp, p.xm));
    float g1 = __fmul_rn(a, __fsub_rn(p.yp, p.ym));
    float g2 = __fmul_rn(a, __fsub_rn(p.zp, p.zm));
    const float dxy1 = __fmul_rn(b, __fsub_rn(p.xpyp, p.xmym)), dxy2 = __fmul_rn(b, __fsub_rn(p.xpym, p.xmyp));
    const float dxz1 = __fmul_rn(b, __fsub_rn(p.xpzp, p.xmzm)), dxz2 = __fmul_rn(b, __fsub_rn(p.xpzm, p.xmzp));
    const float dyz1 = __fmul_rn(b, __fsub_rn(p.ypzp, p.ymzm)), dyz2 = __fmul_rn(b, __fsub_rn(p.ypzm, p.ymzp));
    g0 = __fadd_rn(g0, __fadd_rn(__fadd_rn(__fadd_rn(dxy1, dxy2), dxz1), dxz2));
    g1 = __fadd_rn(g1, __fadd_rn(__fadd_rn(__fsub_rn(dxy1, dxy2), dyz1), dyz2));
    g2 = __fadd_rn(g2, __fsub_rn(__fadd_rn(__fsub_rn(dxz1, dxz2), dyz1), dyz2));
    const float rho_e = __fmul_rn(-k2e, p.c);
    f0 = __fmul_rn(rho_e, __fsub_rn(Ex, g0));
    f1 = __fmul_rn(rho_e, __fsub_rn(Ey, g1));
    f2 = __fmul_rn(rho_e, __fsub_rn(Ez, g2));
}

// host-side split of a double into float-float
__host__ __device__ inline ff ff_from_double(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

}  // namespace es
