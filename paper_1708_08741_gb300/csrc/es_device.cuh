// es_device.cuh -- small device helpers shared by the libes kernels.
#pragma once

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

}  // namespace es
