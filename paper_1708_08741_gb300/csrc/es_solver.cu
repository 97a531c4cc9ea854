// es_solver.cu -- Debye-Hueckel solve (a4, a5) and the EDL field / body force
// (a6); Sec. 4.3, Sec. 5.3, Sec. 5.4, Sec. 5.6.
//
// The 7-point finite-volume stencil of Sec. 4.3 is never stored: an unknown
// cell without the near-boundary bit has the constant stencil
// (6 + kappa^2 h^2, -1 x 6) / h^2; at a near-boundary cell the boundary
// treatment of Sec. 5.4 is applied face by face from the neighbour's kind
// (Dirichlet face: centre +1 and RHS 2 * value; Neumann face: centre -1 and
// RHS sigma / eps; zero-flux wall: centre -1).  This is the quasi-constant
// stencil idea of Sec. 5.3 taken to its limit: one byte per cell.
//
// The outer loop (defect correction) keeps psi and r = b - A psi in FP64,
// or in the MIXED32 form in float-float (two floats, about 48 bits); the
// V-cycle solves A e = r for the correction in the inner type T (double, or
// float in the MIXED32 form).
//
// GB300 executes FP64 arithmetic (and conversions to and from FP64) on a
// pipe with 1/64 of the FP32 rate, so the FP32 kernels here carry no double
// operand at all: level constants come in as T, cell indices are 32-bit
// (N < 2^31), and the MIXED32 body force reads a float copy of psi.
#include <type_traits>

#include "es_device.cuh"

namespace es {

namespace {

constexpr int kRedThreads = 256;

// Programmatic dependent launch for the V-cycle's chain of kernels: a
// kernel launched by launch_pdl may be scheduled while the one before it
// on the stream drains, and waits here (before touching memory) until that
// one has completed and its writes are visible; launched plainly, the wait
// returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
void launch_pdl(const es_ctx* c, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // (errors: cudaGetLastError)
}

__device__ __forceinline__ bool wrap_axis(int v, int n, int per, int& out) {
    if (v < 0 || v >= n) {
        if (!per) return false;
        v = v < 0 ? v + n : v - n;
    }
    out = v;
    return true;
}


template <class T>
struct Level {
    int nx, ny, nz;
    int per[3];
    int pot_bc[6];
    T h2;     // h_l^2
    T diag0;  // 6 + kappa^2 h_l^2
};

// Fine-level face contribution for the FP64 outer residual: adds the centre
// adjustment to diag and the boundary value to b, or returns the index of an
// unknown neighbour (>= 0).
__device__ __forceinline__ int fine_face(const Grid& g, const Solver& s, const int32_t* owner,
                                         const DParticle* part, const int* kind, int x, int y, int z, int a,
                                         int side, double& diag, double& b) {
    int d[3] = {0, 0, 0};
    d[a] = side;
    long long nb;
    if (!neighbour(g, x, y, z, d[0], d[1], d[2], nb)) {
        int face = 2 * a + (side > 0 ? 1 : 0);
        if (s.pot_bc[face] == ES_POT_DIRICHLET) {
            diag += 1.0;
            b += 2.0 * s.pot_val[face];
        } else {
            diag -= 1.0;
        }
        return -1;
    }
    int o = owner[nb];
    if (o < 0) return (int)nb;
    if (kind[o] == ES_KIND_ZETA) {
        diag += 1.0;
        b += 2.0 * part[o].zeta;
    } else {
        diag -= 1.0;
        b += part[o].sigma / s.eps;
    }
    return -1;
}

// r = b - A psi on the unknowns (FP64 form), stored as the V-cycle
// right-hand side, and per-block partial sums of r^2.  Blocks stride over
// rows (y, z); threads over x.  PB: the nonlinear Poisson-Boltzmann form
// (Eq. SPBE): the screening term kappa^2 psi of A psi becomes
// kappa^2 phi_t sinh(psi / phi_t), and the kernel also leaves the shift of
// the stencil's centre entry linearised about psi, kappa^2 (cosh(psi /
// phi_t) - 1), for the sweeps of this iteration (Sec. 5.3: the stencils are
// re-set at the start of every iteration).
template <bool PB>
__global__ void __launch_bounds__(kRedThreads) k_outer_residual(Grid g, Solver s, double diag0, double k2,
                                                                double phi_t, double* __restrict__ dk,
                                                                const double* __restrict__ psi,
                                                                const uint8_t* __restrict__ st0,
                                                                const int32_t* __restrict__ owner,
                                                                const DParticle* __restrict__ part,
                                                                const int* __restrict__ kind,
                                                                double* __restrict__ r_out,
                                                                double* __restrict__ partial) {
    __shared__ double sh[32];
    double acc = 0.0;
    const int nx = g.nx, ny = g.ny, nxy = g.nx * g.ny;
    const int rows = g.ny * g.nz;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = row % ny, z = row / ny;
        const int base = row * nx;
        const int ym = (y == 0 ? ny - 1 : y - 1) - y, yp = (y == ny - 1 ? 0 : y + 1) - y;
        const int zm = (z == 0 ? g.nz - 1 : z - 1) - z, zp = (z == g.nz - 1 ? 0 : z + 1) - z;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const int c = base + x;
            const uint8_t st = st0[c];
            double r = 0.0;
            if ((st & ST_KIND) == ST_UNKNOWN) {
                if (!(st & ST_NEAR)) {
                    const int xm = (x == 0 ? nx - 1 : x - 1) - x, xp = (x == nx - 1 ? 0 : x + 1) - x;
                    double off = psi[c + xm];
                    off += psi[c + xp];
                    off += psi[c + ym * nx];
                    off += psi[c + yp * nx];
                    off += psi[c + zm * nxy];
                    off += psi[c + zp * nxy];
                    r = off - diag0 * psi[c];
                } else {
                    double diag = diag0, b = 0.0, off = 0.0;
                    for (int a = 0; a < 3; a++)
                        for (int side = -1; side <= 1; side += 2) {
                            int nb = fine_face(g, s, owner, part, kind, x, y, z, a, side, diag, b);
                            if (nb >= 0) off += psi[nb];
                        }
                    r = b - (diag * psi[c] - off);
                }
                if constexpr (PB) {
                    const double pc = psi[c], u = pc / phi_t;
                    r += k2 * pc - k2 * phi_t * sinh(u);
                    dk[c] = k2 * (cosh(u) - 1.0);
                }
                acc += r * r;
            }
            r_out[c] = r;
        }
    }
    double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Stores natural cells c .. c+3 (c % 4 == 0, cell c of colour col) of a
// float field in the colour-split layout (cells c, c+2 of colour col sit at
// c/2, c/2+1 of half col; cells c+1, c+3 at the same places of the other).
__device__ __forceinline__ void rb_st4(float* base, int half, int c, int col, float v0, float v1, float v2,
                                       float v3) {
    *reinterpret_cast<float2*>(base + col * half + (c >> 1)) = make_float2(v0, v2);
    *reinterpret_cast<float2*>(base + (col ^ 1) * half + (c >> 1)) = make_float2(v1, v3);
}

// Wall boundary values 2 * pot_val of a Dirichlet wall, as float-float.
struct WallFF {
    float hi[6], lo[6];
};

// r = b - A psi for the MIXED32 form, with psi = psi_hi + psi_lo in
// float-float.  The sum that cancels (neighbours + b - diag * psi_c, whose
// terms are ~1e6 times the residual near convergence) is formed without
// rounding error in its high parts: the diag * psi_c product is split
// exactly with an FMA (TwoProd) and the high parts are accumulated with
// TwoSum, the low parts in plain FP32; the result is then rounded once to
// the float right-hand side of the V-cycles (the only consumer).  The
// diagonal 6 + kappa^2 arrives as float-float; a boundary face changes it
// by +-1 and adds its float-float boundary value to b.  Threads own W = 4
// consecutive cells of a row (16-byte loads, as the vector smoother) or
// single cells (W = 1) when nx is not a multiple of 4; blocks of (32, 8)
// threads stride over z, and each block leaves one partial sum of r^2.
struct HiSum {
    float s, e;  // s + e == exact sum of the high parts added so far (e rounded)
    __device__ __forceinline__ void add(float h) {
        const ff t = two_sum(s, h);
        s = t.hi;
        e = __fadd_rn(e, t.lo);
    }
};

template <int W>
__device__ __forceinline__ void load_span(const float* p, float (&v)[W], int off) {
    if constexpr (W == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[off + 0] = q.x;
        v[off + 1] = q.y;
        v[off + 2] = q.z;
        v[off + 3] = q.w;
    } else {
        v[off] = *p;
    }
}

// Warp-cooperative processing of rare cells.  Lane l marks its cells with
// bit i of `bits` (i < W); the marked cells of the warp are dealt out one per
// lane (in order of i, then of lane), fn(owner_lane, i) computes each one,
// and the value lands in buf[owner_lane * W + i] (a per-warp buffer of
// 32 W floats).  A warp whose near-boundary cells sit at different positions
// of the lanes' spans thus runs the long boundary code once instead of once
// per position.  Every lane of the warp must call this.
template <int W, class V, class Fn>
__device__ __forceinline__ void warp_rare_cells(unsigned bits, V* buf, Fn&& fn) {
    const int lane = threadIdx.x & 31;
    unsigned M[W];
    int P[W + 1];
    P[0] = 0;
#pragma unroll
    for (int i = 0; i < W; i++) {
        M[i] = __ballot_sync(0xffffffffu, (bits >> i) & 1u);
        P[i + 1] = P[i] + __popc(M[i]);
    }
    for (int k0 = 0; k0 < P[W]; k0 += 32) {
        const int k = k0 + lane;
        if (k < P[W]) {
            int i = 0, pi = 0;
            unsigned mi = M[0];
#pragma unroll
            for (int j = 1; j < W; j++)
                if (k >= P[j]) {
                    i = j;
                    pi = P[j];
                    mi = M[j];
                }
            const int owner = (int)__fns(mi, 0, k - pi + 1);
            buf[owner * W + i] = fn(owner, i);
        }
    }
    __syncwarp();
}

// Float-float residual at one near-boundary unknown cell, from global
// memory: faces to unknown cells add the neighbour's psi, faces to sphere
// cells add the sphere's boundary value (b) and move the diagonal by +1
// (Dirichlet) or -1 (Neumann), as read from the neighbour's state byte;
// faces beyond a non-periodic wall do the same with the wall's condition.
__device__ __forceinline__ float near_residual_ff(const Grid& g, ff diag0, const WallFF& wall, int pot_dir_mask,
                                                  const float* __restrict__ psi_hi,
                                                  const float* __restrict__ psi_lo,
                                                  const uint8_t* __restrict__ st0,
                                                  const int32_t* __restrict__ owner,
                                                  const float2* __restrict__ pbc, int x, int y, int z) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int c = x + nx * (y + ny * z);
    HiSum hs = {0.0f, 0.0f};
    float lo = 0.0f;
    int dk = 0;
    const int g3[3] = {x, y, z}, n3[3] = {nx, ny, nz}, stride[3] = {1, nx, nx * ny};
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int ax = k >> 1, side = (k & 1) ? 1 : -1;
        int q = g3[ax] + side;
        if (q < 0 || q >= n3[ax]) {
            if (!g.per[ax]) {
                const int face = 2 * ax + (side > 0 ? 1 : 0);
                if ((pot_dir_mask >> face) & 1) {
                    dk += 1;
                    hs.add(wall.hi[face]);
                    lo = __fadd_rn(lo, wall.lo[face]);
                } else {
                    dk -= 1;
                }
                continue;
            }
            q = q < 0 ? q + n3[ax] : q - n3[ax];
        }
        const int nb = c + (q - g3[ax]) * stride[ax];
        const uint8_t kk = st0[nb] & ST_KIND;
        if (kk == ST_UNKNOWN) {
            hs.add(psi_hi[nb]);
            lo = __fadd_rn(lo, psi_lo[nb]);
        } else {
            dk += kk == ST_DIR ? 1 : -1;
            const float2 bv = pbc[owner[nb]];
            hs.add(bv.x);
            lo = __fadd_rn(lo, bv.y);
        }
    }
    const ff dg = ff_add_f(diag0, (float)dk);
    const float hc = psi_hi[c], lc = psi_lo[c];
    const float p = __fmul_rn(dg.hi, hc);
    float t = __fmaf_rn(dg.hi, hc, -p);
    t = __fmaf_rn(dg.hi, lc, t);
    t = __fmaf_rn(dg.lo, hc, t);
    hs.add(-p);
    lo = __fsub_rn(lo, t);
    return __fadd_rn(hs.s, __fadd_rn(hs.e, lo));
}

// The float-float residual at the near-boundary unknown cells of level 0,
// from the near-cell list (both colours), written to r_out before the main
// pass, which reads them back into its norm sum.
template <class M>
__global__ void __launch_bounds__(256) k_outer_residual_near_ff(Grid g, ff diag0, WallFF wall, int pot_dir_mask,
                                                                const float* __restrict__ psi_hi,
                                                                const float* __restrict__ psi_lo,
                                                                const uint8_t* __restrict__ st0,
                                                                const int32_t* __restrict__ owner,
                                                                const float2* __restrict__ pbc,
                                                                const int* __restrict__ list,
                                                                const int* __restrict__ count, int cap,
                                                                float* __restrict__ r_out, M m) {
    // blockIdx.y: list segment
    const int n = count[blockIdx.y];
    const int* seg = list + (size_t)blockIdx.y * cap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = seg[i];
        const int x = c % g.nx, yz = c / g.nx;
        const int y = yz % g.ny, z = yz / g.ny;
        r_out[m(c, (x + y + z) & 1)] =
            near_residual_ff(g, diag0, wall, pot_dir_mask, psi_hi, psi_lo, st0, owner, pbc, x, y, z);
    }
}

// The interior unknown cells of level 0 (near-boundary cells come from
// k_outer_residual_near_ff, launched just before: the pass reads them back
// into its norm sum).  A thread owns the span xs .. xs+W-1 of row y and
// marches through the planes z0 .. z1-1: the rows (y, z-1), (y, z) and
// (y, z+1) of psi roll through registers, so a plane loads the row
// (y, z+1), the rows (y-1, z) and (y+1, z), two halo values and the state
// bytes, and the loads of plane z+1 are issued before plane z is formed.
// SPLIT: r is stored in the colour-split layout (W == 4).  Each block leaves
// one partial sum of r^2.
template <int W>
struct FFSpan {
    float h[W], l[W];
};

template <int W>
__device__ __forceinline__ void load_ff(FFSpan<W>& s, const float* __restrict__ hi, const float* __restrict__ lo,
                                        int at) {
    load_span<W>(hi + at, s.h, 0);
    load_span<W>(lo + at, s.l, 0);
}

template <int W>
__device__ __forceinline__ unsigned load_states(const uint8_t* __restrict__ st, int at) {
    if constexpr (W == 4)
        return *reinterpret_cast<const unsigned*>(st + at);
    else
        return st[at];
}

template <int W, bool SPLIT>
__global__ void __launch_bounds__(256, 2) k_outer_residual_ff(Grid g, ff diag0, const float* __restrict__ psi_hi,
                                                           const float* __restrict__ psi_lo,
                                                           const uint8_t* __restrict__ st0,
                                                           float* __restrict__ r_out,
                                                           double* __restrict__ partial, int zc,
                                                           const int* __restrict__ gate) {
    static_assert(!SPLIT || W == 4, "the split store takes 4-cell spans");
    if (gate && *gate == 0) return;  // (uniform over the grid: the patched residual runs instead)
    __shared__ float swarp[8];
    const int half = (int)(g.N >> 1);
    float acc = 0.0f;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xs = W * (blockIdx.x * 32 + threadIdx.x);
    const int y = blockIdx.y * 8 + threadIdx.y;
    const bool lane_on = xs < nx;
    const int xq = lane_on ? xs : 0;  // (inactive lanes read a valid span)
    const int z0 = (int)blockIdx.z * zc;
    const int z1 = z0 + zc < nz ? z0 + zc : nz;
    // y is the same for the 32 lanes of a warp, so the march is warp-uniform
    if (y < ny && z0 < z1) {
        // unguarded loads: beyond a wall only near-boundary cells would read,
        // and those are formed from memory by near_residual_ff
        int ym, yp, xl, xr;
        if (!wrap_axis(y - 1, ny, g.per[1], ym)) ym = y;
        if (!wrap_axis(y + 1, ny, g.per[1], yp)) yp = y;
        if (!wrap_axis(xq - 1, nx, g.per[0], xl)) xl = xq;
        if (!wrap_axis(xq + W, nx, g.per[0], xr)) xr = xq;
        // row offsets carried from plane to plane; z + 1 past the last
        // plane is the first (periodic) or the row itself (a wall: any
        // valid row)
        const int plane = nx * ny, back = (nz - 1) * plane, zwall = g.per[2] ? 0 : 1;
        int orow = nx * (y + ny * z0);  // row (y, z)
        int oa = nx * (ym + ny * z0) + xq, ob = nx * (yp + ny * z0) + xq;
        const int dl = xl - xq, dr = xr - xq;
        FFSpan<W> D, X, F, A, B;
        float hlh, hll, hrh, hrl;
        unsigned sv;
        auto load = [&](int z, int row, int a_off, int b_off, FFSpan<W>& f, FFSpan<W>& a, FFSpan<W>& b, float& lh,
                        float& ll, float& rh, float& rl, unsigned& s) {
            const int c0 = row + xq;
            s = load_states<W>(st0, c0);
            load_ff<W>(f, psi_hi, psi_lo, z + 1 < nz ? c0 + plane : (zwall ? c0 : c0 - back));
            load_ff<W>(a, psi_hi, psi_lo, a_off);
            load_ff<W>(b, psi_hi, psi_lo, b_off);
            lh = psi_hi[c0 + dl];
            ll = psi_lo[c0 + dl];
            rh = psi_hi[c0 + dr];
            rl = psi_lo[c0 + dr];
        };
        load_ff<W>(D, psi_hi, psi_lo, z0 > 0 ? orow + xq - plane : (zwall ? orow + xq : orow + xq + back));
        load_ff<W>(X, psi_hi, psi_lo, orow + xq);
        load(z0, orow, oa, ob, F, A, B, hlh, hll, hrh, hrl, sv);
        // (four planes an iteration: the rolled rows are renamed, not moved)
#pragma unroll 4
        for (int z = z0; z < z1; z++) {
            FFSpan<W> nF, nA, nB;
            float nlh = 0.0f, nll = 0.0f, nrh = 0.0f, nrl = 0.0f;
            unsigned nsv = 0;
            if (z + 1 < z1)
                load(z + 1, orow + plane, oa + plane, ob + plane, nF, nA, nB, nlh, nll, nrh, nrl, nsv);
            const int row = orow;
            unsigned near_bits = 0;
            float out[W];
#pragma unroll
            for (int i = 0; i < W; i++) {
                out[i] = 0.0f;
                const unsigned s = lane_on ? (sv >> (8 * i)) & 0xFFu : (unsigned)ST_NEU;
                if ((s & ST_KIND) != ST_UNKNOWN) continue;
                if (s & ST_NEAR) {
                    near_bits |= 1u << i;
                    continue;
                }
                const float hc = X.h[i], lc = X.l[i];
                const float lfh = i == 0 ? hlh : X.h[i - 1], lfl = i == 0 ? hll : X.l[i - 1];
                const float rgh = i == W - 1 ? hrh : X.h[i + 1], rgl = i == W - 1 ? hrl : X.l[i + 1];
                HiSum hs = {0.0f, 0.0f};
                hs.add(lfh);
                hs.add(rgh);
                hs.add(A.h[i]);
                hs.add(B.h[i]);
                hs.add(D.h[i]);
                hs.add(F.h[i]);
                float lo = __fadd_rn(__fadd_rn(__fadd_rn(lfl, rgl), __fadd_rn(A.l[i], B.l[i])),
                                     __fadd_rn(D.l[i], F.l[i]));
                // - diag * psi_c: high product split exactly, low terms to lo
                const float p = __fmul_rn(diag0.hi, hc);
                float t = __fmaf_rn(diag0.hi, hc, -p);
                t = __fmaf_rn(diag0.hi, lc, t);
                t = __fmaf_rn(diag0.lo, hc, t);
                hs.add(-p);
                lo = __fsub_rn(lo, t);
                out[i] = __fadd_rn(hs.s, __fadd_rn(hs.e, lo));
            }
            // near-boundary cells: formed by k_outer_residual_near_ff just before
            const int col0 = (xs + y + z) & 1;
            if (near_bits) {
#pragma unroll
                for (int i = 0; i < W; i++)
                    if ((near_bits >> i) & 1u) {
                        if constexpr (SPLIT)
                            out[i] = r_out[((col0 + i) & 1) * half + ((row + xs + i) >> 1)];
                        else
                            out[i] = r_out[row + xs + i];
                    }
            }
#pragma unroll
            for (int i = 0; i < W; i++) acc = __fmaf_rn(out[i], out[i], acc);
            if (lane_on) {
                if constexpr (SPLIT) {
                    rb_st4(r_out, half, row + xs, col0, out[0], out[1], out[2], out[3]);
                } else if constexpr (W == 4) {
                    *reinterpret_cast<float4*>(r_out + row + xs) = make_float4(out[0], out[1], out[2], out[3]);
                } else {
                    r_out[row + xs] = out[0];
                }
            }
            D = X;
            X = F;
            F = nF;
            A = nA;
            B = nB;
            hlh = nlh;
            hll = nll;
            hrh = nrh;
            hrl = nrl;
            sv = nsv;
            orow += plane;
            oa += plane;
            ob += plane;
        }
    }
    // per-block partial: float within the block (a few thousand terms), one
    // double per block
    float v = acc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) swarp[threadIdx.y] = v;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; w++) tot += (double)swarp[w];
        partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = tot;
    }
}

__global__ void k_finalize_norm(const double* partial, int n, double* out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
    double tot = block_sum(v, sh);
    if (threadIdx.x == 0) out[0] = sqrt(tot);
}

template <class T>
struct Q4 {
    T v0, v1, v2, v3;
};
__device__ __forceinline__ Q4<float> vld(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Q4<double> vld(const double* p) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *(reinterpret_cast<const double2*>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void vst(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void vst(double* p, double a, double b, double c, double d) {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
    *(reinterpret_cast<double2*>(p) + 1) = make_double2(c, d);
}
#define ES_VLD(arr, off, ptr)      \
    do {                           \
        const auto q_ = vld(ptr);  \
        arr[(off) + 0] = q_.v0;    \
        arr[(off) + 1] = q_.v1;    \
        arr[(off) + 2] = q_.v2;    \
        arr[(off) + 3] = q_.v3;    \
    } while (0)

// Loads natural cells c .. c+3 of a float field in the colour-split layout
// (the placement of rb_st4; 8-byte loads).
__device__ __forceinline__ Q4<float> rb_ld4(const float* base, int half, int c, int col) {
    const float2 a = *reinterpret_cast<const float2*>(base + col * half + (c >> 1));
    const float2 b = *reinterpret_cast<const float2*>(base + (col ^ 1) * half + (c >> 1));
    return {a.x, b.x, a.y, b.y};
}

// Access to a level's correction e stored as E: the arithmetic type T
// itself, or (finest level, ES_MG_FP16) FP16 holding s * e, with the scale
// s = sqrt(N) / ||r|| set per correction so that the stored values sit near
// 1 in FP16's normal range; loads return e in T.
template <class T, class E>
struct EAcc;
template <class T>
struct EAcc<T, T> {
    T s, is;
    __device__ __forceinline__ T ld(const T* p) const { return *p; }
    __device__ __forceinline__ void st(T* p, T v) const { *p = v; }
    __device__ __forceinline__ Q4<T> ld4(const T* p) const { return vld(p); }
    __device__ __forceinline__ void st4(T* p, T a, T b, T c, T d) const { vst(p, a, b, c, d); }
};
template <>
struct EAcc<float, __half> {
    float s, is;
    __device__ __forceinline__ float ld(const __half* p) const { return __half2float(*p) * is; }
    __device__ __forceinline__ void st(__half* p, float v) const { *p = __float2half_rn(v * s); }
    __device__ __forceinline__ Q4<float> ld4(const __half* p) const {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return {a.x * is, a.y * is, b.x * is, b.y * is};
    }
    __device__ __forceinline__ void st4(__half* p, float a, float b, float c, float d) const {
        const __half2 h0 = __floats2half2_rn(a * s, b * s), h1 = __floats2half2_rn(c * s, d * s);
        uint2 u;
        u.x = *reinterpret_cast<const unsigned*>(&h0);
        u.y = *reinterpret_cast<const unsigned*>(&h1);
        *reinterpret_cast<uint2*>(p) = u;
    }
};
#define ES_ELD(acc, arr, off, ptr)    \
    do {                              \
        const auto q_ = (acc).ld4(ptr); \
        arr[(off) + 0] = q_.v0;       \
        arr[(off) + 1] = q_.v1;       \
        arr[(off) + 2] = q_.v2;       \
        arr[(off) + 3] = q_.v3;       \
    } while (0)

// Storage index of a level's e and rhs: the natural index (x + nx (y + ny z)),
// or the colour-split layout of the finest level in the reduced forms
// (nx % 8 == 0): the cells of colour (x + y + z) % 2 = k are stored
// contiguously in half k, cell c at k * N/2 + c / 2 (c / 2 = x / 2 +
// nx/2 (y + ny z) for even nx), so that a half sweep streams only its own
// colour and reads the other one.  col is the cell's colour.
struct NatMap {
    __device__ __forceinline__ int operator()(int c, int) const { return c; }
};
struct RbMap {
    int half;
    __device__ __forceinline__ int operator()(int c, int col) const { return col * half + (c >> 1); }
};

// Diagonal and off-diagonal sum of level l at an unknown cell.  With
// READ = false only the diagonal is formed (off = 0, e is not touched).
template <class T, bool READ = true, class E = T, class M = NatMap>
__device__ __forceinline__ void level_stencil(const Level<T>& L, const uint8_t* st, const E* e, int x, int y,
                                              int z, uint8_t s, T& diag, T& off,
                                              const EAcc<T, E>& A = EAcc<T, E>{(T)1, (T)1}, M m = M{}) {
    const int nx = L.nx, nxy = L.nx * L.ny;
    const int c = x + nx * y + nxy * z;
    const int ncol = 1 - ((x + y + z) & 1);  // (the six neighbours have the other colour)
    if (!(s & ST_NEAR)) {
        diag = L.diag0;
        if (!READ) {
            off = (T)0;
            return;
        }
        const int xm = (x == 0 ? nx - 1 : x - 1) - x, xp = (x == nx - 1 ? 0 : x + 1) - x;
        const int ym = (y == 0 ? L.ny - 1 : y - 1) - y, yp = (y == L.ny - 1 ? 0 : y + 1) - y;
        const int zm = (z == 0 ? L.nz - 1 : z - 1) - z, zp = (z == L.nz - 1 ? 0 : z + 1) - z;
        T o = A.ld(e + m(c + xm, ncol));
        o += A.ld(e + m(c + xp, ncol));
        o += A.ld(e + m(c + ym * nx, ncol));
        o += A.ld(e + m(c + yp * nx, ncol));
        o += A.ld(e + m(c + zm * nxy, ncol));
        o += A.ld(e + m(c + zp * nxy, ncol));
        off = o;
        return;
    }
    T dg = L.diag0;
    T o = (T)0;
    const int v[3] = {x, y, z}, n3[3] = {L.nx, L.ny, L.nz}, stride[3] = {1, nx, nxy};
    for (int a = 0; a < 3; a++)
        for (int side = -1; side <= 1; side += 2) {
            int p = v[a] + side;
            if (p < 0 || p >= n3[a]) {
                if (!L.per[a]) {
                    dg += (L.pot_bc[2 * a + (side > 0 ? 1 : 0)] == ES_POT_DIRICHLET) ? (T)1 : (T)-1;
                    continue;
                }
                p = p < 0 ? p + n3[a] : p - n3[a];
            }
            const int nb = c + (p - v[a]) * stride[a];
            const uint8_t k = st[nb] & ST_KIND;
            if (k == ST_UNKNOWN) {
                if (READ) o += A.ld(e + m(nb, ncol));
            } else {
                dg += (k == ST_DIR) ? (T)1 : (T)-1;
            }
        }
    diag = dg;
    off = o;
}

// One red (colour 0) or black (1) Gauss-Seidel / SOR half sweep,
// colour = (i + j + k) mod 2.  Thread t owns the cell pair (2t, 2t+1) of a
// row and updates the one of this colour.  first != 0: the iterate starts
// at zero, so neighbours are not read and the pair's other cell is zeroed.
template <class T>
__global__ void __launch_bounds__(128) k_smooth(Level<T> L, const uint8_t* __restrict__ st,
                                                const T* __restrict__ rhs, T* __restrict__ e, int colour,
                                                int first, T omega, const T* __restrict__ dk = nullptr) {
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (2 * t >= L.nx) return;
    const int par = (colour + y + z) & 1;
    const int x = 2 * t + par;
    const int row = L.nx * (y + L.ny * z);
    if (first && 2 * t + 1 - par < L.nx) e[row + 2 * t + 1 - par] = (T)0;
    if (x >= L.nx) return;  // odd extent: the last pair has one cell
    const int c = row + x;
    const uint8_t s = st[c];
    if ((s & ST_KIND) != ST_UNKNOWN) return;
    T diag, off;
    if (first)
        level_stencil<T, false>(L, st, e, x, y, z, s, diag, off);
    else
        level_stencil<T, true>(L, st, e, x, y, z, s, diag, off);
    if (dk) diag += dk[c];  // (nonlinear Poisson-Boltzmann: the linearised centre entry)
    const T gs = (L.h2 * rhs[c] + off) / diag;
    e[c] = first ? omega * gs : ((T)1 - omega) * e[c] + omega * gs;
}


// The update of the interior cells xs + P0 + 2j of a span (indices known at
// compile time, so the span arrays stay in registers); the near-boundary
// cells of the colour are only marked in near_bits (bit = span position).
template <class T, int P0, int W>
__device__ __forceinline__ void span_update(const Level<T>& L, T inv_diag0, T (&c)[W + 2], const T (&a)[W],
                                            const T (&b)[W], const T (&d)[W], const T (&f)[W], const T (&r)[W],
                                            uint2 sw, T omega, unsigned& near_bits) {
#pragma unroll
    for (int j = 0; j < W / 2; j++) {
        const int i = P0 + 2 * j;
        const uint8_t sv = (uint8_t)(((i < 4 ? sw.x : sw.y) >> (8 * (i & 3))) & 0xFF);
        if ((sv & ST_KIND) != ST_UNKNOWN) continue;
        if (sv & ST_NEAR) {
            near_bits |= 1u << i;
            continue;
        }
        T o = c[i];
        o += c[i + 2];
        o += a[i];
        o += b[i];
        o += d[i];
        o += f[i];
        const T gs = (L.h2 * r[i] + o) * inv_diag0;
        c[i + 1] = ((T)1 - omega) * c[i + 1] + omega * gs;
    }
}

// Gauss-Seidel value of one near-boundary unknown cell of level l, read
// from global memory (the boundary faces per Sec. 5.4 as level_stencil).
// first: 0 the iterate is read; 1 the iterate starts at zero (nothing is
// read); 2 the cell's own old value is zero but its neighbours are read
// (the second colour of a sweep from zero in the colour-split layout).
template <class T, class E = T, class M = NatMap>
__device__ __forceinline__ T near_gs(const Level<T>& L, const uint8_t* __restrict__ st, const T* __restrict__ rhs,
                                     const E* e, int x, int y, int z, int first, T omega,
                                     const EAcc<T, E>& A = EAcc<T, E>{(T)1, (T)1}, M m = M{}) {
    const int cidx = x + L.nx * (y + L.ny * z);
    const int col = (x + y + z) & 1;
    const uint8_t s = st[cidx];
    T diag, off;
    if (first == 1)
        level_stencil<T, false, E, M>(L, st, e, x, y, z, s, diag, off, A, m);
    else
        level_stencil<T, true, E, M>(L, st, e, x, y, z, s, diag, off, A, m);
    const T gs = (L.h2 * rhs[m(cidx, col)] + off) / diag;
    return first ? omega * gs : ((T)1 - omega) * A.ld(e + m(cidx, col)) + omega * gs;
}

// The near-boundary cells of a level, by colour: the level's near-cell list
// and the state bytes their stencils need.
struct NearWork {
    const uint8_t* st;
    const int* list;
    const int* count;
    int cap;
};

// The colour's near-boundary cells of a level shared out to the blocks of a
// half-sweep launch after their interior spans: with at least kNearSegs
// blocks, block b serves segment b % kNearSegs together with the other
// blocks of that residue; with fewer, block b serves segments b, b + nblk, ...
template <class T, class E, class M>
__device__ __forceinline__ void near_share(const Level<T>& L, const NearWork& nw, const T* __restrict__ rhs, E* e,
                                           int colour, int first, T omega, const EAcc<T, E>& A, M m) {
    const int nblk = (int)(gridDim.x * gridDim.y * gridDim.z);
    const int b = ((int)blockIdx.z * (int)gridDim.y + (int)blockIdx.y) * (int)gridDim.x + (int)blockIdx.x;
    const bool many = nblk >= kNearSegs;
    const int tid = (int)((threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x);
    const int nth = (int)(blockDim.x * blockDim.y * blockDim.z);
    for (int seg = many ? b % kNearSegs : b; seg < kNearSegs; seg += many ? kNearSegs : nblk) {
        const int sb = many ? b / kNearSegs : 0;
        const int nsb = many ? (nblk - seg + kNearSegs - 1) / kNearSegs : 1;  // blocks on this segment
        const int k = colour * kNearSegs + seg;
        const int n = nw.count[k];
        const int* list = nw.list + (size_t)k * nw.cap;
        for (int i = sb * nth + tid; i < n; i += nsb * nth) {
            const int cc = list[i];
            const int x = cc % L.nx, yz = cc / L.nx;
            const int yy = yz % L.ny, zz = yz / L.ny;
            A.st(e + m(cc, colour), near_gs<T, E, M>(L, nw.st, rhs, e, x, yy, zz, first, omega, A, m));
        }
    }
}

template <class T, int W, bool INLINE_NEAR, class E = T>
__device__ __forceinline__ void smooth_v_span(const Level<T>& L, T inv_diag0, const uint8_t* __restrict__ st,
                                              const T* __restrict__ rhs, E* __restrict__ e, int colour, int first,
                                              T omega, const EAcc<T, E>& A, int xs, int y, int z);

// One red or black half sweep of a level in the natural layout, 4-cell spans
// (smooth_v_span).  INLINE_NEAR: the colour's near-boundary cells are
// updated inside the spans (small levels); else they come from the level's
// near-cell list, shared out to the same launch's blocks after their spans
// (near_share; both sets read only the other colour, and a span that holds
// a near-boundary cell of the colour stores only its own updates).
template <class T, int W, bool INLINE_NEAR, class E = T>
__global__ void __launch_bounds__(256) k_smooth_v(Level<T> L, T inv_diag0, const uint8_t* __restrict__ st,
                                                  const T* __restrict__ rhs, E* __restrict__ e, int colour,
                                                  int first, T omega, EAcc<T, E> A, NearWork nw) {
    pdl_wait();
    const int xs = W * (blockIdx.x * 32 + threadIdx.x);
    const int y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
    if (y < L.ny) smooth_v_span<T, W, INLINE_NEAR, E>(L, inv_diag0, st, rhs, e, colour, first, omega, A, xs, y, z);
    if constexpr (!INLINE_NEAR) near_share<T, E, NatMap>(L, nw, rhs, e, colour, first, omega, A, NatMap{});
}

template <class T, int W, bool INLINE_NEAR, class E>
__device__ __forceinline__ void smooth_v_span(const Level<T>& L, T inv_diag0, const uint8_t* __restrict__ st,
                                              const T* __restrict__ rhs, E* __restrict__ e, int colour, int first,
                                              T omega, const EAcc<T, E>& A, int xs, int y, int z) {
    static_assert(W == 4, "the near-cell path reads the span's states from one word");
    const bool lane_on = xs < L.nx;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int row = nx * (y + ny * z);
    // Neighbour rows and columns wrap on periodic axes.  Beyond a wall no
    // interior cell reads them (a cell next to a wall is a near-boundary
    // cell, updated from global memory below), so any valid index does
    // there and the loads need no guards.
    int ym, yp, zm, zp, xl, xr;
    if (!wrap_axis(y - 1, ny, L.per[1], ym)) ym = y;
    if (!wrap_axis(y + 1, ny, L.per[1], yp)) yp = y;
    if (!wrap_axis(z - 1, nz, L.per[2], zm)) zm = z;
    if (!wrap_axis(z + 1, nz, L.per[2], zp)) zp = z;
    if (!wrap_axis(xs - 1, nx, L.per[0], xl)) xl = xs;
    if (!wrap_axis(xs + W, nx, L.per[0], xr)) xr = xs;
    const int rym = nx * (ym + ny * z), ryp = nx * (yp + ny * z);
    const int rzm = nx * (y + ny * zm), rzp = nx * (y + ny * zp);
    T c[W + 2], a[W], b[W], d[W], f[W], r[W];
    uint2 sw = make_uint2(0x02020202u, 0x02020202u);  // (Neumann: nothing to update)
    const int xq = lane_on ? xs : 0;                   // (inactive lanes read a valid span)
    if (!first) {
        c[0] = A.ld(e + row + (lane_on ? xl : 0));
        c[W + 1] = A.ld(e + row + (lane_on ? xr : 0));
#pragma unroll
        for (int v = 0; v < W; v += 4) {
            ES_ELD(A, c, 1 + v, e + row + xq + v);
            ES_ELD(A, a, v, e + rym + xq + v);
            ES_ELD(A, b, v, e + ryp + xq + v);
            ES_ELD(A, d, v, e + rzm + xq + v);
            ES_ELD(A, f, v, e + rzp + xq + v);
        }
    } else {
        // the iterate starts at zero
#pragma unroll
        for (int i = 0; i < W + 2; i++) c[i] = (T)0;
#pragma unroll
        for (int i = 0; i < W; i++) a[i] = b[i] = d[i] = f[i] = (T)0;
    }
#pragma unroll
    for (int v = 0; v < W; v += 4) ES_VLD(r, v, rhs + row + xq + v);
    if (lane_on) {
        if (W == 8) {
            sw = *reinterpret_cast<const uint2*>(st + row + xs);
        } else {
            sw.x = *reinterpret_cast<const unsigned*>(st + row + xs);
        }
    }
    const int p0 = (colour + y + z) & 1;  // xs is even: cells xs + p0 + 2j have the colour
    unsigned near_bits = 0;
    if (p0 == 0)
        span_update<T, 0, W>(L, inv_diag0, c, a, b, d, f, r, sw, omega, near_bits);
    else
        span_update<T, 1, W>(L, inv_diag0, c, a, b, d, f, r, sw, omega, near_bits);
    if constexpr (INLINE_NEAR) {
        // Near-boundary cells of the colour, on small levels (where a separate
        // pass would cost more in launch time than it saves): the neighbour
        // values are already in registers; the neighbours' state bytes decide
        // which of them enter the sum and how the diagonal moves (Sec. 5.4:
        // Dirichlet +1, Neumann -1); a face beyond a non-periodic boundary
        // takes the domain condition.  Only warps holding such a cell load
        // the states.
        if (__any_sync(0xffffffffu, near_bits != 0)) {
            const int xq2 = lane_on ? xs : 0;
            const unsigned su = *reinterpret_cast<const unsigned*>(st + rym + xq2);
            const unsigned sd = *reinterpret_cast<const unsigned*>(st + ryp + xq2);
            const unsigned sm = *reinterpret_cast<const unsigned*>(st + rzm + xq2);
            const unsigned sp = *reinterpret_cast<const unsigned*>(st + rzp + xq2);
            const unsigned sl = st[row + (lane_on ? xl : 0)], sr = st[row + (lane_on ? xr : 0)];
            const bool wy0 = !L.per[1] && y == 0, wy1 = !L.per[1] && y == ny - 1;
            const bool wz0 = !L.per[2] && z == 0, wz1 = !L.per[2] && z == nz - 1;
            auto wd = [&](int f) { return L.pot_bc[f] == ES_POT_DIRICHLET ? (T)1 : (T)-1; };
#pragma unroll
            for (int i = 0; i < W; i++) {
                if (!((near_bits >> i) & 1u)) continue;
                const int gx = xs + i;
                T dg = L.diag0, o = (T)0;
                auto face = [&](bool wall, T wdv, unsigned kind, T v) {
                    if (wall)
                        dg += wdv;
                    else if (kind == ST_UNKNOWN)
                        o += v;
                    else
                        dg += kind == ST_DIR ? (T)1 : (T)-1;
                };
                face(!L.per[0] && gx == 0, wd(0), (i == 0 ? sl : (sw.x >> (8 * (i - 1)))) & ST_KIND, c[i]);
                face(!L.per[0] && gx == nx - 1, wd(1), (i == W - 1 ? sr : (sw.x >> (8 * (i + 1)))) & ST_KIND,
                     c[i + 2]);
                face(wy0, wd(2), (su >> (8 * i)) & ST_KIND, a[i]);
                face(wy1, wd(3), (sd >> (8 * i)) & ST_KIND, b[i]);
                face(wz0, wd(4), (sm >> (8 * i)) & ST_KIND, d[i]);
                face(wz1, wd(5), (sp >> (8 * i)) & ST_KIND, f[i]);
                const T gs = (L.h2 * r[i] + o) / dg;
                c[i + 1] = ((T)1 - omega) * c[i + 1] + omega * gs;
            }
        }
    } else {
        // the colour's near-boundary cells belong to the list part of the
        // launch: a span holding one stores only the cells it updated (the
        // colour's interior unknown cells) and, on a sweep from zero, the
        // other colour's zeros (nobody else writes that colour now)
        if (lane_on && near_bits != 0) {
            const int p0 = (colour + y + z) & 1;
#pragma unroll
            for (int i = 0; i < W; i++) {
                const unsigned sv = (sw.x >> (8 * i)) & 0xFFu;
                if ((i & 1) == p0 ? (sv & (ST_KIND | ST_NEAR)) == ST_UNKNOWN : first != 0)
                    A.st(e + row + xs + i, c[1 + i]);
            }
            return;
        }
    }
    if (lane_on) {
#pragma unroll
        for (int v = 0; v < W; v += 4) A.st4(e + row + xs + v, c[1 + v], c[2 + v], c[3 + v], c[4 + v]);
    }
}

// The interior unknown cells of one colour of a colour-split level, for a
// 4-cell span of compact places iq .. iq+3 in row y and the
// planes z0 .. z1-1 (see k_smooth_rb).  The other colour's rows of the
// planes z-1, z and z+1 at row y roll through registers (the row z+1 of one
// plane is the row z of the next and the row z-1 of the one after), so a
// plane loads three new rows of e (z+1, y-1, y+1), one halo value, its
// right-hand side and its mask word; the loads of plane z+1 are issued
// before plane z is updated.  FIRST: 1 the iterate starts at zero (no e is
// read), 2 the colour's old values are zero; GS: omega = 1 (the old value
// is not needed).  A cell's update sums its neighbours in the order of
// k_smooth_v's span_update (x left, x right, y-1, y+1, z-1, z+1), so both
// finest-level layouts give the same bits.
// The row offsets are carried from plane to plane (one add a row a plane),
// the wrap of z + 1 is a select, and the four cells are formed without
// branches (the mask picks the stores only): fewer issued instructions.
template <class T, int FIRST, bool GS>
__device__ __forceinline__ void rb_march(const Level<T>& L, T inv_diag0, const uint32_t* __restrict__ mcol, int wpr,
                                         const T* __restrict__ rcol, const T* __restrict__ eo, T* __restrict__ es,
                                         int colour, T omega, int iq, int y, int z0, int z1) {
    const int nxh = L.nx >> 1, ny = L.ny, nz = L.nz;
    int ym, yp, il, ir;
    if (!wrap_axis(y - 1, ny, L.per[1], ym)) ym = y;
    if (!wrap_axis(y + 1, ny, L.per[1], yp)) yp = y;
    if (!wrap_axis(iq - 1, nxh, L.per[0], il)) il = iq;
    if (!wrap_axis(iq + 4, nxh, L.per[0], ir)) ir = iq;
    const int msh = iq & 31;
    const int plane = nxh * ny, mplane = wpr * ny;
    int oe = nxh * (y + ny * z0) + iq;        // row (y, z): rhs, the other colour, the colour
    int oa = nxh * (ym + ny * z0) + iq;       // row (y-1, z)
    int ob = nxh * (yp + ny * z0) + iq;       // row (y+1, z)
    int om = wpr * (y + ny * z0) + (iq >> 5);  // mask word
    const int hl = il - iq, hr = ir - iq;     // halo offsets in the row
    const int back = (nz - 1) * plane;        // from the last plane to the first
    const int zwall = L.per[2] ? 0 : 1;
    T F[4], A[4], B[4], R[4], h = (T)0;
    unsigned m = 0;
    int O = (colour + y + z0) & 1;
    // plane z's loads; row (y, z+1) is the next plane, or past the last one
    // the first (periodic) or the row itself (a wall)
    auto load = [&](int z, int o, int e_off, int a_off, int b_off, int m_off, T (&f)[4], T (&a)[4], T (&b)[4],
                    T (&r)[4], T& hv, unsigned& mv) {
        mv = (mcol[m_off] >> msh) & 0xFu;
        ES_VLD(r, 0, rcol + e_off);
        if constexpr (FIRST != 1) {
            const int f_off = z + 1 < nz ? e_off + plane : (zwall ? e_off : e_off - back);
            ES_VLD(f, 0, eo + f_off);
            ES_VLD(a, 0, eo + a_off);
            ES_VLD(b, 0, eo + b_off);
            hv = eo[e_off + (o == 0 ? hl : hr)];
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) f[k] = a[k] = b[k] = (T)0;
            hv = (T)0;
        }
    };
    T D[4] = {(T)0, (T)0, (T)0, (T)0}, X[4] = {(T)0, (T)0, (T)0, (T)0};
    if constexpr (FIRST != 1) {
        const int d_off = z0 > 0 ? oe - plane : (zwall ? oe : oe + back);
        ES_VLD(D, 0, eo + d_off);
        ES_VLD(X, 0, eo + oe);
    }
    load(z0, O, oe, oa, ob, om, F, A, B, R, h, m);
    for (int z = z0; z < z1; z++) {
        T nF[4], nA[4], nB[4], nR[4], nh = (T)0;
        unsigned nm = 0;
        if (z + 1 < z1) load(z + 1, O ^ 1, oe + plane, oa + plane, ob + plane, om + mplane, nF, nA, nB, nR, nh, nm);
        if (m) {
            T C[4] = {(T)0, (T)0, (T)0, (T)0};
            if constexpr (FIRST == 0 && !GS) ES_VLD(C, 0, es + oe);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const T left = O == 0 ? (k == 0 ? h : X[k - 1]) : X[k];
                const T right = O == 0 ? X[k] : (k == 3 ? h : X[k + 1]);
                T o = left;
                o += right;
                o += A[k];
                o += B[k];
                o += D[k];
                o += F[k];
                const T gs = (L.h2 * R[k] + o) * inv_diag0;
                if constexpr (FIRST != 0)
                    C[k] = omega * gs;
                else if constexpr (GS)
                    C[k] = gs;
                else
                    C[k] = ((T)1 - omega) * C[k] + omega * gs;
            }
            if (m == 0xFu) {
                vst(es + oe, C[0], C[1], C[2], C[3]);
            } else {
                // (the colour's near-boundary cells belong to the near blocks)
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if ((m >> k) & 1u) es[oe + k] = C[k];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            D[k] = X[k];
            X[k] = F[k];
            F[k] = nF[k];
            A[k] = nA[k];
            B[k] = nB[k];
            R[k] = nR[k];
        }
        h = nh;
        m = nm;
        O ^= 1;
        oe += plane;
        oa += plane;
        ob += plane;
        om += mplane;
    }
}

// One red (colour 0) or black (1) half sweep of the finest level in the
// colour-split layout (reduced forms, nx % 8 == 0), interior and
// near-boundary cells in one launch.  The two sets are disjoint and both
// read only the other colour, so they need no order:
//  * a thread owns 4 consecutive compact places of the colour in one row
//    (8 natural cells) and marches through zc planes (rb_march), loading
//    the other colour's rows and its right-hand side as 16-byte vectors and
//    storing the cells it updates.  Which cells those are (the interior
//    unknown cells) it reads from the colour's bit mask (one bit per cell,
//    rows padded to whole 32-bit words), not from the state bytes.  A
//    Gauss-Seidel update (omega = 1) does not need the cell's old value, so
//    the colour's own e is read only for omega != 1;
//  * then every block takes its share of the colour's near-boundary cells
//    from the near-cell list (Gauss-Seidel values with the boundary faces of
//    Sec. 5.4, near_gs): about half a cell per thread on large
//    grids, whose scattered, latency-bound loads overlap the streaming of
//    the blocks still marching.
// Per cell and half sweep the interior moves the other colour's e in, the
// colour's e out and its rhs in: 6 bytes, plus 1/16 byte of mask (against 9
// with the state bytes and the colour's old values, and 13 in the
// interleaved layout).  Cells that are not unknown are never written: no
// kernel reads e there.  Same per-cell arithmetic as k_smooth_v.  first: 1
// the iterate starts at zero (nothing is read), 2 the colour's old values
// are zero (the second colour of a sweep from zero).  Four blocks per SM:
// the register cap keeps enough loads in flight to stream at the HBM rate.
template <class T>
__global__ void __launch_bounds__(256, 4) k_smooth_rb(Level<T> L, T inv_diag0, const uint32_t* __restrict__ mask,
                                                      int wpr, const T* __restrict__ rhs, T* __restrict__ e,
                                                      int colour, int first, T omega, int half, NearWork nw,
                                                      int zc) {
    pdl_wait();
    const int i0 = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int y = blockIdx.y * 8 + threadIdx.y;
    if (y < L.ny && i0 < (L.nx >> 1)) {
        const int z0 = (int)blockIdx.z * zc;
        const int z1 = z0 + zc < L.nz ? z0 + zc : L.nz;
        const uint32_t* mcol = mask + (size_t)colour * ((size_t)L.ny * L.nz * wpr);
        const T* rcol = rhs + (size_t)colour * half;
        const T* eo = e + (size_t)(colour ^ 1) * half;
        T* es = e + (size_t)colour * half;
        if (first == 1)
            rb_march<T, 1, false>(L, inv_diag0, mcol, wpr, rcol, eo, es, colour, omega, i0, y, z0, z1);
        else if (first == 2)
            rb_march<T, 2, false>(L, inv_diag0, mcol, wpr, rcol, eo, es, colour, omega, i0, y, z0, z1);
        else if (omega == (T)1)
            rb_march<T, 0, true>(L, inv_diag0, mcol, wpr, rcol, eo, es, colour, omega, i0, y, z0, z1);
        else
            rb_march<T, 0, false>(L, inv_diag0, mcol, wpr, rcol, eo, es, colour, omega, i0, y, z0, z1);
    }
    // the near-boundary cells, shared out to the blocks
    near_share<T, T, RbMap>(L, nw, rhs, e, colour, first, omega, EAcc<T, T>{(T)1, (T)1}, RbMap{half});
}

__device__ __forceinline__ bool axis_ok(int v, int n, int per, int& w) {
    if (v >= 0 && v < n) {
        w = v;
        return true;
    }
    if (!per) return false;
    w = v % n;
    if (w < 0) w += n;
    return true;
}

// ---- fused red-black sweep, span form ----
//
// One full Gauss-Seidel sweep (red half, then black half) in a single pass
// over the level, out of place (ein -> eout; no block writes what another
// reads, so blocks never wait on one another).  A block marches up z: at
// plane p it updates the red cells of plane p on its tile plus a one-cell
// ring, then the black cells of plane p - 1 on the tile (all of whose red
// neighbours are final by then), and writes plane p - 1.  Per cell and sweep
// the level moves e in and out once, plus rhs and the state byte: half the
// traffic of two in-place half sweeps.  Layout as in the vector smoother: lane l of row-warp w owns the 4-cell span x0 + 4l .. +3
// of row y0 - 2 + w, so a block covers 128 x cells and 16 rows, of which
// rows 2..13 are written (rows 1 and 14 get red updates only, rows 0 and 15
// are loaded only).  Planes stream into a 7-slot shared-memory ring with
// cp.async, three planes ahead; the x neighbours just outside the tile
// (x0 - 1 and x0 + 128) are updated by a 17th "ring" warp, one lane per row
// and side.  Interior cells use 16-byte shared loads; near-boundary cells
// read the neighbour states from the ring as well.  Requires nx % 128 == 0.
constexpr int kRbRows = 16, kRbOut = 12, kRbSpans = 34, kRbSlots = 7;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(pred ? 16 : 0));
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool pred) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(pred ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;\n" ::); }

// ---- finest-level half sweep staged by bulk asynchronous copies ----
//
// mbarrier and bulk-copy primitives (sm_90 and later).  A wait is bounded:
// after about a second it reports failure and the kernel records
// DS_TIMEOUT instead of spinning on.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1LL << 31)) return false;  // (about a second)
    return true;
}
// bytes from global src to shared dst (both 16-byte aligned, bytes a
// multiple of 16), completing on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Tile of the staged half sweep: a block owns whole compact rows (nxh
// cells of one colour, tpr = nxh / 4 threads a row, 4 cells a thread) of ty
// rows and marches through zc planes; kBulkSlots ring slots each hold one
// plane of the other colour's rows y0 - 1 .. y0 + ty (the y halo) and one
// plane of the colour's right-hand side rows.
constexpr int kBulkSlots = 6;
struct BulkShape {
    int tpr, ty, zc;
};

// One half sweep of the interior unknown cells of a tile (see
// k_smooth_rb_bulk).  Stage k of the pipeline brings the other colour's
// plane z0 - 1 + k and the right-hand side of plane z0 - 2 + k into slot
// k % kBulkSlots; plane z0 + j is updated once stages j, j + 1, j + 2 have
// landed (the other colour below, at and above it, its rhs), and its slot j
// is refilled with stage j + kBulkSlots after the block's barrier.  FIRST
// and GS as in rb_march, the same per-cell arithmetic (and so the same bits).
// Returns false when a wait timed out (the copies still in flight have
// been waited for, with the same bound).
template <class T, int FIRST, bool GS>
__device__ bool rb_bulk_march(const Level<T>& L, T inv_diag0, const uint32_t* __restrict__ mcol, int wpr,
                              const T* __restrict__ rcol, const T* __restrict__ eo, T* __restrict__ es, T omega,
                              int colour, const BulkShape& B, int y0, int z0, int z1, T* slots, uint64_t* bars) {
    const int nxh = L.nx >> 1, ny = L.ny, nz = L.nz;
    const int W = nxh, TY = B.ty;
    const int tyc = y0 + TY <= ny ? TY : ny - y0;  // rows of this tile
    const int zc = z1 - z0, nstage = zc + 2;
    const size_t slot_floats = (size_t)(2 * TY + 2) * W;
    auto wrap_y = [&](int y) {
        int w;
        if (!wrap_axis(y, ny, L.per[1], w)) w = y < 0 ? 0 : ny - 1;  // (beyond a wall: any valid row)
        return w;
    };
    auto wrap_z = [&](int z) {
        int w;
        if (!wrap_axis(z, nz, L.per[2], w)) w = z < 0 ? 0 : nz - 1;
        return w;
    };
    // the producer: one thread issues a stage's bulk copies
    auto issue = [&](int k) {
        T* base = slots + (size_t)(k % kBulkSlots) * slot_floats;
        uint64_t* bar = bars + (k % kBulkSlots);
        const int zr = z0 - 2 + k;
        const bool has_r = k >= 2 && zr < z1;
        const unsigned rowb = (unsigned)W * sizeof(T);
        unsigned bytes = 0;
        if (FIRST != 1) bytes += (unsigned)(tyc + 2) * rowb;
        if (has_r) bytes += (unsigned)tyc * rowb;
        mbar_expect_tx(bar, bytes);
        if (FIRST != 1) {
            const int zo = wrap_z(z0 - 1 + k);
            const T* pl = eo + (size_t)nxh * ny * zo;
            bulk_g2s(base, pl + (size_t)nxh * wrap_y(y0 - 1), rowb, bar);
            bulk_g2s(base + W, pl + (size_t)nxh * y0, (unsigned)tyc * rowb, bar);
            bulk_g2s(base + (size_t)(tyc + 1) * W, pl + (size_t)nxh * wrap_y(y0 + tyc), rowb, bar);
        }
        if (has_r) bulk_g2s(base + (size_t)(TY + 2) * W, rcol + (size_t)nxh * (y0 + (size_t)ny * zr), (unsigned)tyc * rowb, bar);
    };
    const int t = threadIdx.x;
    const int ty = t / B.tpr, iq = 4 * (t % B.tpr);
    const bool on = ty < tyc;
    const int y = y0 + (on ? ty : 0);
    int il, ir;
    if (!wrap_axis(iq - 1, nxh, L.per[0], il)) il = iq;
    if (!wrap_axis(iq + 4, nxh, L.per[0], ir)) ir = iq;
    if (t == 0)
        for (int k = 0; k < kBulkSlots && k < nstage; k++) issue(k);
    // this thread's mask word of plane z (loaded a plane ahead)
    auto mask_word = [&](int z) { return on ? mcol[(size_t)wpr * (y + (size_t)ny * z) + (iq >> 5)] : 0u; };
    unsigned mw = mask_word(z0);
    int waited = 0;  // stages waited for
    bool ok = true;
    int j = 0;       // planes done
    for (; j < zc && ok; j++) {
        const unsigned mw_next = j + 1 < zc ? mask_word(z0 + j + 1) : 0u;
        while (waited <= j + 2 && ok) {
            ok = mbar_wait(bars + (waited % kBulkSlots), (unsigned)((waited / kBulkSlots) & 1));
            if (ok) waited++;
        }
        if (!ok) break;
        const int z = z0 + j;
        const T* sA = slots + (size_t)(j % kBulkSlots) * slot_floats;        // other colour, z - 1
        const T* sB = slots + (size_t)((j + 1) % kBulkSlots) * slot_floats;  // other colour, z
        const T* sC = slots + (size_t)((j + 2) % kBulkSlots) * slot_floats;  // other colour z + 1, rhs z
        const unsigned m = (mw >> (iq & 31)) & 0xFu;
        mw = mw_next;
        if (m) {
            T X[4], A[4], Bv[4], D[4], F[4], R[4], h = (T)0;
            const int O = (colour + y + z) & 1;
            if constexpr (FIRST != 1) {
                ES_VLD(X, 0, sB + (size_t)(ty + 1) * W + iq);
                ES_VLD(A, 0, sB + (size_t)ty * W + iq);
                ES_VLD(Bv, 0, sB + (size_t)(ty + 2) * W + iq);
                ES_VLD(D, 0, sA + (size_t)(ty + 1) * W + iq);
                ES_VLD(F, 0, sC + (size_t)(ty + 1) * W + iq);
                h = sB[(size_t)(ty + 1) * W + (O == 0 ? il : ir)];
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) X[k] = A[k] = Bv[k] = D[k] = F[k] = (T)0;
            }
            ES_VLD(R, 0, sC + (size_t)(TY + 2) * W + (size_t)ty * W + iq);
            T C[4] = {(T)0, (T)0, (T)0, (T)0};
            const size_t rz = (size_t)nxh * (y + (size_t)ny * z) + iq;
            if constexpr (FIRST == 0 && !GS) ES_VLD(C, 0, es + rz);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (!((m >> k) & 1u)) continue;
                T left, right;
                if (O == 0) {
                    left = k == 0 ? h : X[k - 1];
                    right = X[k];
                } else {
                    left = X[k];
                    right = k == 3 ? h : X[k + 1];
                }
                T o = left;
                o += right;
                o += A[k];
                o += Bv[k];
                o += D[k];
                o += F[k];
                const T gs = (L.h2 * R[k] + o) * inv_diag0;
                if constexpr (FIRST != 0)
                    C[k] = omega * gs;
                else if constexpr (GS)
                    C[k] = gs;
                else
                    C[k] = ((T)1 - omega) * C[k] + omega * gs;
            }
            if (m == 0xFu) {
                vst(es + rz, C[0], C[1], C[2], C[3]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if ((m >> k) & 1u) es[rz + k] = C[k];
            }
        }
        __syncthreads();  // (every thread is done with slot j % kBulkSlots)
        if (t == 0 && j + kBulkSlots < nstage) issue(j + kBulkSlots);
    }
    if (!ok) {
        // the copies already issued (the prologue's stages and one more per
        // plane done) must land before the block leaves
        const int issued = nstage < kBulkSlots + j ? nstage : kBulkSlots + j;
        for (int k = waited; k < issued; k++) mbar_wait(bars + (k % kBulkSlots), (unsigned)((k / kBulkSlots) & 1));
    }
    return ok;
}

// The colour-split finest level's half sweep with the other colour's rows
// and the colour's right-hand side staged in shared memory by bulk
// asynchronous copies (nx / 2 <= 256 compact cells a row): one thread of a
// block issues a plane's copies -- a few contiguous row runs, kilobytes each --
// three planes ahead of the update, so the loads in flight no longer depend
// on the registers of the threads; the update reads its neighbours from
// shared memory.  Moves the same 6.06 bytes a cell as k_smooth_rb, computes
// the same bits, and afterwards takes its share of the colour's
// near-boundary cells as k_smooth_rb does.  A wait that runs out sets
// DS_TIMEOUT in status and the block skips the rest.
template <class T>
__global__ void __launch_bounds__(256) k_smooth_rb_bulk(Level<T> L, T inv_diag0, const uint32_t* __restrict__ mask,
                                                        int wpr, const T* __restrict__ rhs, T* __restrict__ e,
                                                        int colour, int first, T omega, int half, NearWork nw,
                                                        BulkShape B, int* status) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ __align__(8) uint64_t bars[kBulkSlots];
    T* slots = (T*)bsm;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kBulkSlots; k++) mbar_init(bars + k, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int y0 = (int)blockIdx.x * B.ty;
    const int z0 = (int)blockIdx.y * B.zc;
    const int z1 = z0 + B.zc < L.nz ? z0 + B.zc : L.nz;
    const uint32_t* mcol = mask + (size_t)colour * ((size_t)L.ny * L.nz * wpr);
    const T* rcol = rhs + (size_t)colour * half;
    const T* eo = e + (size_t)(colour ^ 1) * half;
    T* es = e + (size_t)colour * half;
    bool ok;
    if (first == 1)
        ok = rb_bulk_march<T, 1, false>(L, inv_diag0, mcol, wpr, rcol, eo, es, omega, colour, B, y0, z0, z1, slots,
                                        bars);
    else if (first == 2)
        ok = rb_bulk_march<T, 2, false>(L, inv_diag0, mcol, wpr, rcol, eo, es, omega, colour, B, y0, z0, z1, slots,
                                        bars);
    else if (omega == (T)1)
        ok = rb_bulk_march<T, 0, true>(L, inv_diag0, mcol, wpr, rcol, eo, es, omega, colour, B, y0, z0, z1, slots,
                                       bars);
    else
        ok = rb_bulk_march<T, 0, false>(L, inv_diag0, mcol, wpr, rcol, eo, es, omega, colour, B, y0, z0, z1, slots,
                                        bars);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(status, DS_TIMEOUT);
        return;
    }
    // the colour's near-boundary cells, shared out as in k_smooth_rb
    near_share<T, T, RbMap>(L, nw, rhs, e, colour, first, omega, EAcc<T, T>{(T)1, (T)1}, RbMap{half});
}

template <class T>
struct RB2 {
    using Span = T[4];
    static constexpr size_t e_bytes = (size_t)kRbSlots * kRbRows * kRbSpans * 4 * sizeof(T);
    static constexpr size_t s_bytes = (size_t)kRbSlots * kRbRows * kRbSpans * 4;
    static constexpr size_t smem = e_bytes + s_bytes;
};

// Gauss-Seidel value of one cell from the shared-memory ring, any stencil:
// jc, jm, jp index the cell in the slots of planes z, z - 1, z + 1 (the
// state of element j is byte j & 3 of word j >> 2 of the state ring); bit f
// of `wall` marks face f (x-, x+, y-, y+, z-, z+) as beyond a non-periodic
// boundary, where the face condition of the potential applies instead.
template <class T>
__device__ __forceinline__ T rb2_near(const Level<T>& L, T omega, const T* __restrict__ E,
                                      const unsigned* __restrict__ S, int jc, int jm, int jp, T rhsv,
                                      unsigned wall) {
    constexpr int ROW = kRbSpans * 4;
    const int nb[6] = {jc - 1, jc + 1, jc - ROW, jc + ROW, jm, jp};
    T dg = L.diag0, o = (T)0;
#pragma unroll
    for (int f = 0; f < 6; f++) {
        if ((wall >> f) & 1u) {
            dg += (L.pot_bc[f] == ES_POT_DIRICHLET) ? (T)1 : (T)-1;
            continue;
        }
        const int j = nb[f];
        const unsigned kind = (S[j >> 2] >> ((j & 3) << 3)) & ST_KIND;
        if (kind == ST_UNKNOWN)
            o += E[j];
        else
            dg += (kind == ST_DIR) ? (T)1 : (T)-1;
    }
    const T gs = (L.h2 * rhsv + o) / dg;
    return ((T)1 - omega) * E[jc] + omega * gs;
}

// Faces of cell (gx, gy, gz) that lie beyond a non-periodic boundary.
template <class T>
__device__ __forceinline__ unsigned wall_faces(const Level<T>& L, int gx, int gy, int gz) {
    unsigned m = 0;
    if (!L.per[0]) m |= (gx == 0 ? 1u : 0u) | (gx == L.nx - 1 ? 2u : 0u);
    if (!L.per[1]) m |= (gy == 0 ? 4u : 0u) | (gy == L.ny - 1 ? 8u : 0u);
    if (!L.per[2]) m |= (gz == 0 ? 16u : 0u) | (gz == L.nz - 1 ? 32u : 0u);
    return m;
}

template <class T>
__global__ void __launch_bounds__(32 * (kRbRows + 1), sizeof(T) == 4 ? 2 : 1) k_smooth_rb2(Level<T> L, T inv_diag0,
                                                                  const uint8_t* __restrict__ st,
                                                                  const T* __restrict__ rhs,
                                                                  const T* __restrict__ ein, T* __restrict__ eout,
                                                                  int first, T omega, int zc) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char rb2_smem[];
    __shared__ T sbuf[kRbRows][32 * 4];
    constexpr int SE = kRbRows * kRbSpans * 4;  // elements of one plane slot
    constexpr int SS = kRbRows * kRbSpans;      // state words of one plane slot
    constexpr int ROW = kRbSpans * 4;           // elements of one ring row
    T* E = reinterpret_cast<T*>(rb2_smem);
    unsigned* S = reinterpret_cast<unsigned*>(rb2_smem + RB2<T>::e_bytes);
    const int lane = threadIdx.x, w = threadIdx.y;
    const bool ring = w == kRbRows;
    const int nx = L.nx, ny = L.ny, nz = L.nz, nxy = nx * ny;
    const int x0 = blockIdx.x * 128, y0 = blockIdx.y * kRbOut;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
    // what this thread loads: a row warp its span of row w, the ring warp the
    // left (lanes 0-15) or right ring span of row lane % 16
    const int lrow = ring ? (lane & 15) : w;
    const int lspan = ring ? ((lane >> 4) ? kRbSpans - 1 : 0) : lane + 1;
    const int lidx = lrow * kRbSpans + lspan;
    int gy_l = 0, gx_l = 0;
    const bool xy_ok = axis_ok(y0 - 2 + lrow, ny, L.per[1], gy_l) && axis_ok(x0 - 4 + 4 * lspan, nx, L.per[0], gx_l);
    const int goff = gx_l + nx * gy_l;
    auto wrap7 = [](int v) { return v >= kRbSlots ? v - kRbSlots : (v < 0 ? v + kRbSlots : v); };
    auto plane = [&](int p, int& gz) { return axis_ok(p, nz, L.per[2], gz); };
    auto issue = [&](int p, int sl) {
        int gz = 0;
        const bool ok = xy_ok && p <= z1 + 1 && plane(p, gz);
        const int off = ok ? goff + nxy * gz : 0;
        T* de = E + sl * SE + lidx * 4;
#pragma unroll
        for (int h = 0; h < (int)(4 * sizeof(T) / 16); h++)
            cp_async16(reinterpret_cast<unsigned char*>(de) + 16 * h,
                       reinterpret_cast<const unsigned char*>(ein + off) + 16 * h, ok && !first);
        cp_async4(S + sl * SS + lidx, st + off, ok);
        cp_async_commit();
    };
    // right-hand sides in registers, two planes ahead: a row warp keeps its
    // span, the ring warp the one cell it updates
    const int rk = ring ? ((lane >> 4) ? 128 : -1) : 4 * lane;
    int rgx = 0;
    const bool rx_ok = axis_ok(x0 + rk, nx, L.per[0], rgx);
    auto fetch_rhs = [&](int p, T (&r)[4]) {
        int gz = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) r[i] = (T)0;
        if (!(p >= z0 - 1 && p <= z1 && xy_ok && plane(p, gz))) return;
        const T* src = rhs + (nxy * gz + nx * gy_l);
        if (!ring) {
            const auto q = vld(src + x0 + rk);
            r[0] = q.v0;
            r[1] = q.v1;
            r[2] = q.v2;
            r[3] = q.v3;
        } else if (rx_ok) {
            r[0] = src[rgx];
        }
    };
    T r_m1[4], r_0[4], r_p1[4], r_p2[4];
    for (int p = z0 - 2; p <= z0 + 1; p++) issue(p, wrap7(p - z0 + 3));
    fetch_rhs(z0 - 1, r_0);
    fetch_rhs(z0, r_p1);
#pragma unroll
    for (int i = 0; i < 4; i++) r_m1[i] = (T)0;

    const int ry = y0 - 2 + w;  // row of a row warp (unwrapped)
    int gry = 0;
    const bool row_ok = !ring && axis_ok(ry, ny, L.per[1], gry);
    const bool red_row = row_ok && w >= 1 && w <= kRbRows - 2;
    const bool out_row = !ring && w >= 2 && w < 2 + kRbOut && ry < ny;
    const int own = (w * kRbSpans + lane + 1) * 4;  // own span, element offset within a slot
    T* buf = sbuf[ring ? 0 : w];
    int sl = 2;  // slot of plane p (p = z0 - 1)
    for (int p = z0 - 1; p <= z1; p++) {
        const int s_m2 = wrap7(sl - 2), s_m1 = wrap7(sl - 1), s_p1 = wrap7(sl + 1);
        issue(p + 3, wrap7(sl + 3));
        fetch_rhs(p + 2, r_p2);
        cp_async_wait2();
        __syncthreads();
        int gz = 0;
        const bool zok = plane(p, gz);
        // red cells of plane p: rows 1..14 and the ring cells
        if (!ring) {
            unsigned near = 0;
            const int jc = sl * SE + own;
            if (zok && red_row) {
                const auto c = vld(E + jc);
                const T cm = E[jc - 1], cp = E[jc + 4];
                const auto u = vld(E + jc - ROW);
                const auto d = vld(E + jc + ROW);
                const auto zm = vld(E + s_m1 * SE + own);
                const auto zp = vld(E + s_p1 * SE + own);
                const unsigned sw = S[jc >> 2];
                const T cc[6] = {cm, c.v0, c.v1, c.v2, c.v3, cp};
                const T uu[4] = {u.v0, u.v1, u.v2, u.v3}, dd[4] = {d.v0, d.v1, d.v2, d.v3};
                const T mm[4] = {zm.v0, zm.v1, zm.v2, zm.v3}, pp[4] = {zp.v0, zp.v1, zp.v2, zp.v3};
                const int p0 = (ry + p) & 1;  // red cells at span positions p0 and p0 + 2
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    if ((i & 1) != p0) continue;
                    const unsigned sv = (sw >> (8 * i)) & 0xFFu;
                    if ((sv & ST_KIND) != ST_UNKNOWN) continue;
                    if (sv & ST_NEAR) {
                        near |= 1u << i;
                        continue;
                    }
                    T o = cc[i];
                    o += cc[i + 2];
                    o += uu[i];
                    o += dd[i];
                    o += mm[i];
                    o += pp[i];
                    const T gs = (L.h2 * r_0[i] + o) * inv_diag0;
                    E[jc + i] = ((T)1 - omega) * cc[i + 1] + omega * gs;
                }
            }
            if (__any_sync(0xffffffffu, near != 0)) {
                const int jw = sl * SE + w * ROW + 4, jwm = s_m1 * SE + w * ROW + 4, jwp = s_p1 * SE + w * ROW + 4;
                warp_rare_cells<4>(near, buf, [&](int ln, int i) {
                    const int k = 4 * ln + i;
                    return rb2_near<T>(L, omega, E, S, jw + k, jwm + k, jwp + k,
                                       rhs[nxy * gz + nx * gry + x0 + k], wall_faces(L, x0 + k, gry, gz));
                });
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if ((near >> i) & 1u) E[jc + i] = buf[lane * 4 + i];
            }
        } else if (zok) {
            const int rw = lane & 15, k = rk;
            const int yy = y0 - 2 + rw;
            int gyy = 0;
            if (rw >= 1 && rw <= kRbRows - 2 && rx_ok && axis_ok(yy, ny, L.per[1], gyy) &&
                ((x0 + k + yy + p) & 1) == 0) {
                const int jc = sl * SE + rw * ROW + k + 4;
                const unsigned sv = (S[jc >> 2] >> ((jc & 3) << 3)) & 0xFFu;
                if ((sv & ST_KIND) == ST_UNKNOWN)
                    E[jc] = rb2_near<T>(L, omega, E, S, jc, s_m1 * SE + rw * ROW + k + 4, s_p1 * SE + rw * ROW + k + 4,
                                        r_0[0], wall_faces(L, rgx, gyy, gz));
            }
        }
        __syncthreads();
        // black cells of plane p - 1 on the output rows, then the span out
        const int pb = p - 1;
        if (out_row && pb >= z0 && pb < z1) {  // warp-uniform
            const int jc = s_m1 * SE + own;
            const auto c = vld(E + jc);
            const T cm = E[jc - 1], cp = E[jc + 4];
            const auto u = vld(E + jc - ROW);
            const auto d = vld(E + jc + ROW);
            const auto zm = vld(E + s_m2 * SE + own);
            const auto zp = vld(E + sl * SE + own);
            const unsigned sw = S[jc >> 2];
            const T cc[6] = {cm, c.v0, c.v1, c.v2, c.v3, cp};
            const T uu[4] = {u.v0, u.v1, u.v2, u.v3}, dd[4] = {d.v0, d.v1, d.v2, d.v3};
            const T mm[4] = {zm.v0, zm.v1, zm.v2, zm.v3}, pp[4] = {zp.v0, zp.v1, zp.v2, zp.v3};
            T out[4] = {c.v0, c.v1, c.v2, c.v3};
            unsigned near = 0;
            const int p0 = (ry + pb + 1) & 1;  // black cells at span positions p0 and p0 + 2
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if ((i & 1) != p0) continue;
                const unsigned sv = (sw >> (8 * i)) & 0xFFu;
                if ((sv & ST_KIND) != ST_UNKNOWN) continue;
                if (sv & ST_NEAR) {
                    near |= 1u << i;
                    continue;
                }
                T o = cc[i];
                o += cc[i + 2];
                o += uu[i];
                o += dd[i];
                o += mm[i];
                o += pp[i];
                const T gs = (L.h2 * r_m1[i] + o) * inv_diag0;
                out[i] = ((T)1 - omega) * cc[i + 1] + omega * gs;
            }
            if (__any_sync(0xffffffffu, near != 0)) {
                const int jw = s_m1 * SE + w * ROW + 4, jwm = s_m2 * SE + w * ROW + 4, jwp = sl * SE + w * ROW + 4;
                warp_rare_cells<4>(near, buf, [&](int ln, int i) {
                    const int k = 4 * ln + i;
                    return rb2_near<T>(L, omega, E, S, jw + k, jwm + k, jwp + k, rhs[nxy * pb + nx * ry + x0 + k],
                                       wall_faces(L, x0 + k, ry, pb));
                });
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if ((near >> i) & 1u) out[i] = buf[lane * 4 + i];
            }
            vst(eout + (nxy * pb + nx * ry + x0 + rk), out[0], out[1], out[2], out[3]);
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            r_m1[i] = r_0[i];
            r_0[i] = r_p1[i];
            r_p1[i] = r_p2[i];
        }
        sl = s_p1;
    }
    asm volatile("cp.async.wait_all;\n" ::);
}

// Residual of level l at its unknown cells, restricted to level l+1 as the
// mean of the 8 children (children that are not unknowns contribute 0).
template <class T>
__global__ void __launch_bounds__(128) k_residual_restrict(Level<T> L, const uint8_t* __restrict__ st,
                                                           const T* __restrict__ rhs, const T* __restrict__ e,
                                                           int cnx, int cny, const uint8_t* __restrict__ cst,
                                                           T* __restrict__ crhs) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= cnx) return;
    T sum = (T)0;
    for (int dk = 0; dk < 2; dk++)
        for (int dj = 0; dj < 2; dj++)
            for (int di = 0; di < 2; di++) {
                const int x = 2 * i + di, y = 2 * j + dj, z = 2 * k + dk;
                const int c = x + L.nx * (y + L.ny * z);
                const uint8_t s = st[c];
                T r = (T)0;
                if ((s & ST_KIND) == ST_UNKNOWN) {
                    T diag, off;
                    level_stencil<T>(L, st, e, x, y, z, s, diag, off);
                    const T Ae = (diag * e[c] - off) / L.h2;
                    r = rhs[c] - Ae;
                }
                sum += r;
            }
    const int C = i + cnx * (j + cny * k);
    crhs[C] = ((cst[C] & ST_KIND) == ST_UNKNOWN) ? sum / (T)8 : (T)0;
}

// e_l += e_{l+1}(parent) at unknown cells whose parent is an unknown
// (piecewise-constant prolongation).
template <class T>
__global__ void __launch_bounds__(128) k_prolong(Level<T> L, const uint8_t* __restrict__ st, T* __restrict__ e,
                                                 int cnx, int cny, const uint8_t* __restrict__ cst,
                                                 const T* __restrict__ ce) {
    pdl_wait();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const int c = x + L.nx * (y + L.ny * z);
    const int C = (x >> 1) + cnx * ((y >> 1) + cny * (z >> 1));
    if ((st[c] & ST_KIND) == ST_UNKNOWN && (cst[C] & ST_KIND) == ST_UNKNOWN) e[c] += ce[C];
}

// Vectorized prolongation: a thread owns 4 fine cells of a row (nx % 4 == 0)
// and adds the correction of their 2 parents.
// SPLIT: e of this level colour-split (half: half its cells); chalf != 0:
// the coarse e colour-split too (chalf: half the coarse cells).  C is even,
// so C and C + 1 sit at place C / 2 of their colours.
template <class T, class E, bool SPLIT = false>
__global__ void __launch_bounds__(256) k_prolong_v(Level<T> L, const uint8_t* __restrict__ st, E* __restrict__ e,
                                                   int cnx, int cny, const uint8_t* __restrict__ cst,
                                                   const T* __restrict__ ce, EAcc<T, E> A, int half = 0,
                                                   int chalf = 0) {
    pdl_wait();
    const int xs = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
    if (xs >= L.nx || y >= L.ny) return;
    const int c = xs + L.nx * (y + L.ny * z);
    const int C = (xs >> 1) + cnx * ((y >> 1) + cny * (z >> 1));
    const unsigned sw = *reinterpret_cast<const unsigned*>(st + c);
    const uint8_t c0 = cst[C] & ST_KIND, c1 = cst[C + 1] & ST_KIND;
    T e0, e1;
    if (chalf) {
        const int cc = ((xs >> 1) + (y >> 1) + (z >> 1)) & 1;
        e0 = ce[cc * chalf + (C >> 1)];
        e1 = ce[(cc ^ 1) * chalf + (C >> 1)];
    } else {
        e0 = ce[C];
        e1 = ce[C + 1];
    }
    const int col0 = (xs + y + z) & 1;
    Q4<T> q;
    if constexpr (SPLIT)
        q = rb_ld4(e, half, c, col0);
    else
        q = A.ld4(e + c);
    T v[4] = {q.v0, q.v1, q.v2, q.v3};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint8_t sv = (uint8_t)((sw >> (8 * i)) & ST_KIND);
        const uint8_t pk = i < 2 ? c0 : c1;
        if (sv == ST_UNKNOWN && pk == ST_UNKNOWN) v[i] += i < 2 ? e0 : e1;
    }
    if constexpr (SPLIT)
        rb_st4(e, half, c, col0, v[0], v[1], v[2], v[3]);
    else
        A.st4(e + c, v[0], v[1], v[2], v[3]);
}

// Stores coarse cells C .. C+3 (C % 4 == 0, the first of colour col) of a
// right-hand side: natural order, or colour-split when chalf (half the
// coarse level's cells) is not 0.
__device__ __forceinline__ void store_coarse4(float* __restrict__ crhs, int C, int col, int chalf,
                                              const float (&v)[4]) {
    if (chalf)
        rb_st4(crhs, chalf, C, col, v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<float4*>(crhs + C) = make_float4(v[0], v[1], v[2], v[3]);
}

// Prolongation onto a colour-split level ahead of a Gauss-Seidel
// post-smoothing (omega = 1): the red half sweep that follows replaces each
// red unknown cell without reading it, so only the black cells -- the
// neighbours it reads -- take the correction (e += e_{l+1}(parent) at
// unknown cells whose parent is unknown, as k_prolong_v); the red cells
// keep a stale value until that sweep overwrites them.  A thread owns the
// black compact cells X0 .. X0+3 of one row (natural x = 2X + O,
// O = (1 + y + z) & 1), whose parents are the consecutive coarse cells
// X0 .. X0+3 of coarse row (y/2, z/2).  chalf != 0: the coarse e
// colour-split (chalf: half the coarse cells).
__global__ void __launch_bounds__(256) k_prolong_black_rb(Level<float> L, const uint8_t* __restrict__ st,
                                                          float* __restrict__ e, int half, int cnx, int cny,
                                                          const uint8_t* __restrict__ cst,
                                                          const float* __restrict__ ce, int chalf) {
    pdl_wait();
    const int nxh = L.nx >> 1;
    const int X0 = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
    if (X0 >= nxh || y >= L.ny) return;
    const int O = (1 + y + z) & 1;
    float* eb = e + half + nxh * (y + L.ny * z) + X0;
    const uint2 sw = *reinterpret_cast<const uint2*>(st + L.nx * (y + L.ny * z) + 2 * X0);
    const int C = X0 + cnx * ((y >> 1) + cny * (z >> 1));
    const uchar4 cs = *reinterpret_cast<const uchar4*>(cst + C);
    const uint8_t ck[4] = {cs.x, cs.y, cs.z, cs.w};
    float cv[4];
    if (chalf) {
        const Q4<float> q = rb_ld4(ce, chalf, C, (X0 + (y >> 1) + (z >> 1)) & 1);
        cv[0] = q.v0;
        cv[1] = q.v1;
        cv[2] = q.v2;
        cv[3] = q.v3;
    } else {
        ES_VLD(cv, 0, ce + C);
    }
    float v[4];
    ES_VLD(v, 0, eb);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int j = 2 * k + O;  // natural offset of the black cell in the 8-cell span
        const unsigned sv = ((j < 4 ? sw.x : sw.y) >> (8 * (j & 3))) & ST_KIND;
        if (sv == ST_UNKNOWN && (ck[k] & ST_KIND) == ST_UNKNOWN) v[k] += cv[k];
    }
    vst(eb, v[0], v[1], v[2], v[3]);
}

// Vectorized residual + restriction: a thread owns 2 coarse cells of a
// coarse row, i.e. a 4 x 2 x 2 block of fine cells (nx % 4 == 0).  For each
// of its 4 fine rows it loads the row (with one cell of x halo from the
// neighbouring vectors) and the 4 neighbour rows as 16-byte vectors, forms
// the residuals and adds them to the coarse sums in the children order
// (dk, dj, di) of the scalar kernel.
template <class T, class E = T, class M = NatMap>
__device__ __forceinline__ T near_residual(const Level<T>& L, const uint8_t* __restrict__ st,
                                           const T* __restrict__ rhs, const E* __restrict__ e, int x, int y, int z,
                                           T inv_h2, const EAcc<T, E>& A = EAcc<T, E>{(T)1, (T)1}, M m = M{}) {
    const int cidx = x + L.nx * (y + L.ny * z);
    const int sc = m(cidx, (x + y + z) & 1);
    T diag, off;
    level_stencil<T, true, E, M>(L, st, e, x, y, z, st[cidx], diag, off, A, m);
    return rhs[sc] - (diag * A.ld(e + sc) - off) * inv_h2;
}

// The residual at the near-boundary unknown cells of a level, from its
// near-cell list (both colours), into a scratch array that the restriction
// then reads for those children.
template <class T, class E, class M = NatMap>
__global__ void __launch_bounds__(256) k_near_residual(Level<T> L, const uint8_t* __restrict__ st,
                                                       const T* __restrict__ rhs, const E* __restrict__ e,
                                                       const int* __restrict__ list, const int* __restrict__ count,
                                                       int cap, T inv_h2, T* __restrict__ out, EAcc<T, E> A,
                                                       M m = M{}) {
    pdl_wait();
    // blockIdx.y: list segment
    const int n = count[blockIdx.y];
    const int* seg = list + (size_t)blockIdx.y * cap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = seg[i];
        const int x = c % L.nx, yz = c / L.nx;
        out[c] = near_residual<T, E, M>(L, st, rhs, e, x, yz % L.ny, yz / L.ny, inv_h2, A, m);  // (natural)
    }
}

// SPLIT: e and rhs of this level in the colour-split layout (float).
template <class T, class E, bool SPLIT = false>
__global__ void __launch_bounds__(256) k_restrict_v(Level<T> L, T inv_diag0, T inv_h2, const uint8_t* __restrict__ st,
                                                    const T* __restrict__ rhs, const E* __restrict__ e,
                                                    const T* __restrict__ near_res, int cnx,
                                                    int cny, const uint8_t* __restrict__ cst, T* __restrict__ crhs,
                                                    EAcc<T, E> A, int half = 0, int red_only = 0) {
    pdl_wait();
    const int cx_warp = 2 * (blockIdx.x * 32);
    const int cxs = cx_warp + 2 * threadIdx.x;
    const int cy = blockIdx.y * 8 + threadIdx.y, cz = blockIdx.z;
    if (cy >= cny) return;  // whole warps
    const bool lane_on = cxs < cnx;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int xs = 2 * cxs;
    T sum0 = (T)0, sum1 = (T)0;
#pragma unroll
    for (int dk = 0; dk < 2; dk++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++) {
            const int y = 2 * cy + dj, z = 2 * cz + dk;
            const int row = nx * (y + ny * z);
            // unguarded loads, as in k_smooth_v: beyond a wall only
            // near-boundary cells would read, and those come from memory below
            int ym, yp, zm, zp, xl, xr;
            if (!wrap_axis(y - 1, ny, L.per[1], ym)) ym = y;
            if (!wrap_axis(y + 1, ny, L.per[1], yp)) yp = y;
            if (!wrap_axis(z - 1, nz, L.per[2], zm)) zm = z;
            if (!wrap_axis(z + 1, nz, L.per[2], zp)) zp = z;
            const int xq = lane_on ? xs : 0;
            if (!wrap_axis(xq - 1, nx, L.per[0], xl)) xl = xq;
            if (!wrap_axis(xq + 4, nx, L.per[0], xr)) xr = xq;
            const int rym = nx * (ym + ny * z), ryp = nx * (yp + ny * z);
            const int rzm = nx * (y + ny * zm), rzp = nx * (y + ny * zp);
            T c[6], a[4], b[4], d[4], f[4], r[4];
            if constexpr (SPLIT) {
                static_assert(std::is_same<T, float>::value && std::is_same<E, float>::value, "float split layout");
                const RbMap mp{half};
                const int yz = y + z, col0 = (xq + yz) & 1;
                c[0] = e[mp(row + xl, (xl + yz) & 1)];
                c[5] = e[mp(row + xr, (xr + yz) & 1)];
                auto put = [](T* v, int o, Q4<T> q) {
                    v[o] = q.v0;
                    v[o + 1] = q.v1;
                    v[o + 2] = q.v2;
                    v[o + 3] = q.v3;
                };
                put(c, 1, rb_ld4(e, half, row + xq, col0));
                put(a, 0, rb_ld4(e, half, rym + xq, (xq + ym + z) & 1));
                put(b, 0, rb_ld4(e, half, ryp + xq, (xq + yp + z) & 1));
                put(d, 0, rb_ld4(e, half, rzm + xq, (xq + y + zm) & 1));
                put(f, 0, rb_ld4(e, half, rzp + xq, (xq + y + zp) & 1));
                put(r, 0, rb_ld4(rhs, half, row + xq, col0));
            } else {
                c[0] = A.ld(e + row + xl);
                c[5] = A.ld(e + row + xr);
                ES_ELD(A, c, 1, e + row + xq);
                ES_ELD(A, a, 0, e + rym + xq);
                ES_ELD(A, b, 0, e + ryp + xq);
                ES_ELD(A, d, 0, e + rzm + xq);
                ES_ELD(A, f, 0, e + rzp + xq);
                ES_VLD(r, 0, rhs + row + xq);
            }
            const unsigned sw = lane_on ? *reinterpret_cast<const unsigned*>(st + row + xs) : 0x02020202u;
            T res[4];
            unsigned near_bits = 0;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint8_t sv = (uint8_t)((sw >> (8 * i)) & 0xFF);
                res[i] = (T)0;
                if ((sv & ST_KIND) != ST_UNKNOWN) continue;
                if (sv & ST_NEAR) {
                    near_bits |= 1u << i;
                    continue;
                }
                T o = c[i];
                o += c[i + 2];
                o += a[i];
                o += b[i];
                o += d[i];
                o += f[i];
                res[i] = r[i] - (L.diag0 * c[i + 1] - o) * inv_h2;
            }
            // near-boundary children: formed by k_near_residual just before
#pragma unroll
            for (int i = 0; i < 4; i++)
                if ((near_bits >> i) & 1u) res[i] = near_res[row + xq + i];
            if (red_only) {
                // (after a Gauss-Seidel black half sweep the black residuals
                // vanish: see k_restrict_red_rb)
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if ((xq + i + y + z) & 1) res[i] = (T)0;
            }
            sum0 += res[0] + res[1];
            sum1 += res[2] + res[3];
        }
    if (!lane_on) return;
    const int C = cxs + cnx * (cy + cny * cz);
    const T v0 = ((cst[C] & ST_KIND) == ST_UNKNOWN) ? sum0 / (T)8 : (T)0;
    const T v1 = ((cst[C + 1] & ST_KIND) == ST_UNKNOWN) ? sum1 / (T)8 : (T)0;
    crhs[C] = v0;
    crhs[C + 1] = v1;
    (void)inv_diag0;
}

// Residual + restriction from the colour-split finest level (float,
// nx % 8 == 0).  A block of 32 x 8 threads covers 128 coarse cells of two
// coarse rows; the 4 warps of a coarse row take one fine row of the
// children each (threadIdx.y = 4 * row + 2 dk + dj), so a thread forms the
// residuals of 8 fine cells: in a fine row, the two children of coarse
// cell X are the compact cells X of the two colours (x = 2X and 2X+1), so
// it loads 4 compact cells of each colour, the same places of the four
// neighbour rows (where the colours swap), one halo value per colour and
// the right-hand sides, all as 16-byte vectors.  The four partial sums of
// a coarse cell are then added through shared memory in the order of
// k_restrict_v (dk outer, dj inner), whose arithmetic this repeats exactly;
// near-boundary children come from k_near_residual.
__global__ void __launch_bounds__(256) k_restrict_rb(Level<float> L, float inv_h2, const uint8_t* __restrict__ st,
                                                     const float* __restrict__ rhs, const float* __restrict__ e,
                                                     const float* __restrict__ near_res, int cnx, int cny,
                                                     const uint8_t* __restrict__ cst, float* __restrict__ crhs,
                                                     int half, int chalf) {
    pdl_wait();
    __shared__ float4 part[8][32];
    const int X0 = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int crow = threadIdx.y >> 2, sub = threadIdx.y & 3;
    const int cy = blockIdx.y * 2 + crow, cz = blockIdx.z;
    const bool row_on = cy < cny;
    const bool lane_on = X0 < cnx && row_on;
    const int Xq = X0 < cnx ? X0 : 0;
    const int cyq = row_on ? cy : 0;  // (rows past the end compute on a valid row; nothing is stored)
    const int nx = L.nx, ny = L.ny, nz = L.nz, nxh = nx >> 1;
    const int dk = sub >> 1, dj = sub & 1;
    const int y = 2 * cyq + dj, z = 2 * cz + dk;
    int ym, yp, zm, zp, il, ir;
    if (!wrap_axis(y - 1, ny, L.per[1], ym)) ym = y;
    if (!wrap_axis(y + 1, ny, L.per[1], yp)) yp = y;
    if (!wrap_axis(z - 1, nz, L.per[2], zm)) zm = z;
    if (!wrap_axis(z + 1, nz, L.per[2], zp)) zp = z;
    if (!wrap_axis(Xq - 1, nxh, L.per[0], il)) il = Xq;
    if (!wrap_axis(Xq + 4, nxh, L.per[0], ir)) ir = Xq;
    const int pe = (y + z) & 1;  // colour of the even-x cells of this row
    const float* E0 = e + pe * half;        // x = 2X of this row; x = 2X + 1 of the neighbour rows
    const float* E1 = e + (pe ^ 1) * half;  // x = 2X + 1 of this row; x = 2X of the neighbour rows
    const int rowh = nxh * (y + ny * z);
    const int hym = nxh * (ym + ny * z), hyp = nxh * (yp + ny * z);
    const int hzm = nxh * (y + ny * zm), hzp = nxh * (y + ny * zp);
    float A[4], B[4], r[4], a[4], b[4], d[4], f[4];
    ES_VLD(A, 0, E0 + rowh + Xq);
    ES_VLD(B, 0, E1 + rowh + Xq);
    const float hl = E1[rowh + il], hr = E0[rowh + ir];
    const uint2 sw = *reinterpret_cast<const uint2*>(st + nx * (y + ny * z) + 2 * Xq);
    float res[8];
    // even-x children (A): x neighbours B[k-1] (or the halo), B[k]
    ES_VLD(r, 0, rhs + pe * half + rowh + Xq);
    ES_VLD(a, 0, E1 + hym + Xq);
    ES_VLD(b, 0, E1 + hyp + Xq);
    ES_VLD(d, 0, E1 + hzm + Xq);
    ES_VLD(f, 0, E1 + hzp + Xq);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const unsigned sv = ((k < 2 ? sw.x : sw.y) >> (16 * (k & 1))) & 0xFFu;
        res[2 * k] = 0.0f;
        if ((sv & (ST_KIND | ST_NEAR)) != ST_UNKNOWN) continue;
        float o = k == 0 ? hl : B[k - 1];
        o += B[k];
        o += a[k];
        o += b[k];
        o += d[k];
        o += f[k];
        res[2 * k] = r[k] - (L.diag0 * A[k] - o) * inv_h2;
    }
    // odd-x children (B): x neighbours A[k], A[k+1] (or the halo)
    ES_VLD(r, 0, rhs + (pe ^ 1) * half + rowh + Xq);
    ES_VLD(a, 0, E0 + hym + Xq);
    ES_VLD(b, 0, E0 + hyp + Xq);
    ES_VLD(d, 0, E0 + hzm + Xq);
    ES_VLD(f, 0, E0 + hzp + Xq);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const unsigned sv = ((k < 2 ? sw.x : sw.y) >> (16 * (k & 1) + 8)) & 0xFFu;
        res[2 * k + 1] = 0.0f;
        if ((sv & (ST_KIND | ST_NEAR)) != ST_UNKNOWN) continue;
        float o = A[k];
        o += k == 3 ? hr : A[k + 1];
        o += a[k];
        o += b[k];
        o += d[k];
        o += f[k];
        res[2 * k + 1] = r[k] - (L.diag0 * B[k] - o) * inv_h2;
    }
    // near-boundary children: formed by k_near_residual just before
    const int rown = nx * (y + ny * z) + 2 * Xq;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const unsigned sv = ((j < 4 ? sw.x : sw.y) >> (8 * (j & 3))) & 0xFFu;
        if ((sv & (ST_KIND | ST_NEAR)) == (ST_UNKNOWN | ST_NEAR)) res[j] = near_res[rown + j];
    }
    part[threadIdx.y][threadIdx.x] = make_float4(res[0] + res[1], res[2] + res[3], res[4] + res[5], res[6] + res[7]);
    __syncthreads();
    if (sub != 0 || !lane_on) return;
    float sum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < 4; q++) {  // q = 2 dk + dj: dk outer, dj inner
        const float4 p = part[4 * crow + q][threadIdx.x];
        sum[0] += p.x;
        sum[1] += p.y;
        sum[2] += p.z;
        sum[3] += p.w;
    }
    const int C = X0 + cnx * (cy + cny * cz);
    const uchar4 cs = *reinterpret_cast<const uchar4*>(cst + C);
    const uint8_t ck[4] = {cs.x, cs.y, cs.z, cs.w};
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = ((ck[k] & ST_KIND) == ST_UNKNOWN) ? sum[k] / 8.0f : 0.0f;
    store_coarse4(crhs, C, (X0 + cy + cz) & 1, chalf, v);
}

// The residual of the corrected potential on the colour-split finest level
// (reduced forms), r <- r - A e in FP32, formed by updating the previous
// residual instead of recomputing b - A psi (psi += e is k_correct_ff's).
// A e h^2 = sum over the faces of (e_c - e_nb) + kappa^2 h^2 e_c: the
// differences carry no rounding of the smooth part of e, which dominates e
// near convergence (|e| up to 1/kappa^2 times |r|).  A thread owns 8
// natural cells of a row (the compact cells X0 .. X0+3 of both colours) and
// marches through the planes z0 .. z1-1: the even- and odd-x cells of the
// rows (y, z-1), (y, z) and (y, z+1) roll through registers, so a plane
// loads the row (y, z+1), the rows (y-1, z) and (y+1, z), r, two halo
// values and the state bytes, and the loads of plane z+1 are issued before
// plane z is formed.  Near-boundary cells take r - A e from
// k_near_residual's scratch (natural index); other cells keep r = 0.  Each
// block leaves one partial sum of r^2.
// CORRECT: the same pass applies the correction psi += e (float-float, at
// unknown cells, as k_correct_ff) to the 8 natural cells of each plane it
// forms, so e and the state bytes are read once for both.
template <bool CORRECT>
__global__ void __launch_bounds__(256, 2) k_residual_update_rb(Level<float> L, float inv_h2,
                                                               const uint8_t* __restrict__ st,
                                                               float* __restrict__ rhs, const float* __restrict__ e,
                                                               const float* __restrict__ near_res, int half,
                                                               double* __restrict__ partial, int zc,
                                                               float* __restrict__ psi_hi, float* __restrict__ psi_lo) {
    __shared__ float swarp[8];
    const int nx = L.nx, ny = L.ny, nz = L.nz, nxh = nx >> 1;
    const int X0 = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int y = blockIdx.y * 8 + threadIdx.y;
    const bool lane_on = X0 < nxh;
    const int Xq = lane_on ? X0 : 0;
    const float k2h2 = L.diag0 - 6.0f;  // (exact: diag0 in [6, 12))
    const int z0 = (int)blockIdx.z * zc;
    const int z1 = z0 + zc < nz ? z0 + zc : nz;
    float acc = 0.0f;
    if (y < ny && z0 < z1) {
        int ym, yp, il, ir;
        if (!wrap_axis(y - 1, ny, L.per[1], ym)) ym = y;
        if (!wrap_axis(y + 1, ny, L.per[1], yp)) yp = y;
        if (!wrap_axis(Xq - 1, nxh, L.per[0], il)) il = Xq;
        if (!wrap_axis(Xq + 4, nxh, L.per[0], ir)) ir = Xq;
        // row offsets carried from plane to plane (compact rows: rowh, y -+ 1;
        // natural: the state bytes); z + 1 past the last plane is the first
        // (periodic) or the row itself (a wall: any valid row, only
        // near-boundary cells would read it)
        const int plane = nxh * ny, back = (nz - 1) * plane, zwall = L.per[2] ? 0 : 1;
        int orh = nxh * (y + ny * z0) + Xq, oym = nxh * (ym + ny * z0) + Xq, oyp = nxh * (yp + ny * z0) + Xq;
        int ost = nx * (y + ny * z0) + 2 * Xq;
        const int dl = il - Xq, dr = ir - Xq;
        // plane z's loads: the even- and odd-x cells of row (y, z+1), the
        // rows (y -+ 1, z) of both arrays, r of both colours, the halos
        // and the state bytes.  E0 holds the cells of colour (y + z) & 1 of
        // row (y, z), the even-x ones.
        float Fe[4], Fo[4], a1[4], b1[4], a0[4], b0[4], rE[4], rO[4], hl, hr;
        uint2 sw;
        auto load = [&](int z, int rh, int hm, int hp, int so, float (&fe)[4], float (&fo)[4], float (&pa1)[4],
                        float (&pb1)[4], float (&pa0)[4], float (&pb0)[4], float (&re)[4], float (&ro)[4], float& l,
                        float& r, uint2& s) {
            const int pe = (y + z) & 1;
            const float* E0 = e + pe * half;
            const float* E1 = e + (pe ^ 1) * half;
            const int hzp = z + 1 < nz ? rh + plane : (zwall ? rh : rh - back);
            s = *reinterpret_cast<const uint2*>(st + so);
            ES_VLD(fe, 0, E1 + hzp);
            ES_VLD(fo, 0, E0 + hzp);
            ES_VLD(pa1, 0, E1 + hm);
            ES_VLD(pb1, 0, E1 + hp);
            ES_VLD(pa0, 0, E0 + hm);
            ES_VLD(pb0, 0, E0 + hp);
            ES_VLD(re, 0, rhs + pe * half + rh);
            ES_VLD(ro, 0, rhs + (pe ^ 1) * half + rh);
            l = E1[rh + dl];
            r = E0[rh + dr];
        };
        // the even (De, Ae) and odd (Do, Ao) cells of rows (y, z0-1), (y, z0)
        float De[4], Do[4], Ae[4], Ao[4];
        {
            const int pe = (y + z0) & 1;
            const int hzm = z0 > 0 ? orh - plane : (zwall ? orh : orh + back);
            ES_VLD(De, 0, e + (pe ^ 1) * half + hzm);
            ES_VLD(Do, 0, e + pe * half + hzm);
            ES_VLD(Ae, 0, e + pe * half + orh);
            ES_VLD(Ao, 0, e + (pe ^ 1) * half + orh);
        }
        load(z0, orh, oym, oyp, ost, Fe, Fo, a1, b1, a0, b0, rE, rO, hl, hr, sw);
        for (int z = z0; z < z1; z++) {
            float nFe[4], nFo[4], na1[4], nb1[4], na0[4], nb0[4], nrE[4], nrO[4], nhl = 0.0f, nhr = 0.0f;
            uint2 nsw = make_uint2(0u, 0u);
            if (z + 1 < z1)
                load(z + 1, orh + plane, oym + plane, oyp + plane, ost + nx * ny, nFe, nFo, na1, nb1, na0, nb0, nrE,
                     nrO, nhl, nhr, nsw);
            const int pe = (y + z) & 1;
            const int rowh = orh - Xq, rown = ost;
            float out[8];
            unsigned near = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const unsigned sv = ((k < 2 ? sw.x : sw.y) >> (16 * (k & 1))) & 0xFFu;
                out[2 * k] = rE[k];  // (0 at non-unknown cells)
                if ((sv & ST_KIND) != ST_UNKNOWN) continue;
                if (sv & ST_NEAR) {
                    near |= 1u << (2 * k);
                    continue;
                }
                const float ec = Ae[k];
                float o = ec - (k == 0 ? hl : Ao[k - 1]);
                o += ec - Ao[k];
                o += ec - a1[k];
                o += ec - b1[k];
                o += ec - De[k];
                o += ec - Fe[k];
                o += k2h2 * ec;
                out[2 * k] = rE[k] - o * inv_h2;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const unsigned sv = ((k < 2 ? sw.x : sw.y) >> (16 * (k & 1) + 8)) & 0xFFu;
                out[2 * k + 1] = rO[k];
                if ((sv & ST_KIND) != ST_UNKNOWN) continue;
                if (sv & ST_NEAR) {
                    near |= 1u << (2 * k + 1);
                    continue;
                }
                const float ec = Ao[k];
                float o = ec - Ae[k];
                o += ec - (k == 3 ? hr : Ae[k + 1]);
                o += ec - a0[k];
                o += ec - b0[k];
                o += ec - Do[k];
                o += ec - Fo[k];
                o += k2h2 * ec;
                out[2 * k + 1] = rO[k] - o * inv_h2;
            }
            // near-boundary cells from the scratch
            if (near) {
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if ((near >> j) & 1u) out[j] = near_res[rown + j];
            }
            if (lane_on) {
#pragma unroll
                for (int j = 0; j < 8; j++) acc = __fmaf_rn(out[j], out[j], acc);
                vst(rhs + pe * half + rowh + X0, out[0], out[2], out[4], out[6]);
                vst(rhs + (pe ^ 1) * half + rowh + X0, out[1], out[3], out[5], out[7]);
                if constexpr (CORRECT) {
                    // natural cells 2 X0 .. 2 X0 + 7: e of the even cells is Ae, of the odd ones Ao
                    float hv[8], lv[8];
                    ES_VLD(hv, 0, psi_hi + rown);
                    ES_VLD(hv, 4, psi_hi + rown + 4);
                    ES_VLD(lv, 0, psi_lo + rown);
                    ES_VLD(lv, 4, psi_lo + rown + 4);
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const unsigned sv = ((j < 4 ? sw.x : sw.y) >> (8 * (j & 3))) & 0xFFu;
                        if ((sv & ST_KIND) != ST_UNKNOWN) continue;
                        const ff v = ff_add_f({hv[j], lv[j]}, (j & 1) ? Ao[j >> 1] : Ae[j >> 1]);
                        hv[j] = v.hi;
                        lv[j] = v.lo;
                    }
                    vst(psi_hi + rown, hv[0], hv[1], hv[2], hv[3]);
                    vst(psi_hi + rown + 4, hv[4], hv[5], hv[6], hv[7]);
                    vst(psi_lo + rown, lv[0], lv[1], lv[2], lv[3]);
                    vst(psi_lo + rown + 4, lv[4], lv[5], lv[6], lv[7]);
                }
            }
            // plane z+1's even cells are the odd-colour array of row z's
            // parity, so the roll keeps the even / odd roles
#pragma unroll
            for (int k = 0; k < 4; k++) {
                De[k] = Ae[k];
                Do[k] = Ao[k];
                Ae[k] = Fe[k];
                Ao[k] = Fo[k];
                Fe[k] = nFe[k];
                Fo[k] = nFo[k];
                a1[k] = na1[k];
                b1[k] = nb1[k];
                a0[k] = na0[k];
                b0[k] = nb0[k];
                rE[k] = nrE[k];
                rO[k] = nrO[k];
            }
            hl = nhl;
            hr = nhr;
            sw = nsw;
            orh += plane;
            oym += plane;
            oyp += plane;
            ost += nx * ny;
        }
    }
    float v = acc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) swarp[threadIdx.y] = v;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; w++) tot += (double)swarp[w];
        partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = tot;
    }
}

// Residual + restriction right after a black Gauss-Seidel half sweep
// (omega = 1) on a colour-split level.  That half sweep solved every black
// cell's equation exactly for the red values around it, which it does not
// change, so the black residuals vanish (up to rounding) and the restricted
// residual is the mean of the 4 red children's residuals (the 4 black
// children count as 0).  A thread forms the residuals of the red compact
// cells X0 .. X0+3 of fine row y (the red children of coarse cells X0 ..
// X0+3) and marches up the fine planes 2 cz0 .. 2 cz1 - 1: the black rows
// (y, z-1), (y, z) and (y, z+1) roll through registers, so a plane loads
// the black rows (y, z+1), (y-1, z) and (y+1, z), one halo value, the red
// e and rhs of (y, z) and the state bytes (about 7 bytes per fine cell),
// and the loads of plane z+1 are issued before plane z is formed.  The two
// warps of a coarse row (dj = 0, 1) meet in shared memory after each pair
// of fine planes, and the 4 red children are added in the order of
// k_restrict_v (dk outer, dj inner).  Near-boundary red children come from
// k_near_residual (red segments).  chalf != 0: the coarse right-hand side
// is stored colour-split (chalf: half the coarse cells).
constexpr int kRestrictRows = 4;  // coarse rows per block (2 warps each)

__global__ void __launch_bounds__(32 * 2 * kRestrictRows)
    k_restrict_red_rb(Level<float> L, float inv_h2, const uint8_t* __restrict__ st, const float* __restrict__ rhs,
                      const float* __restrict__ e, const float* __restrict__ near_res, int cnx, int cny, int cnz,
                      const uint8_t* __restrict__ cst, float* __restrict__ crhs, int half, int chalf, int czc) {
    pdl_wait();
    __shared__ float4 part[2][kRestrictRows][4][32];  // (coarse-plane parity, coarse row, 2 dk + dj, lane)
    const int nxh = L.nx >> 1, ny = L.ny, nz = L.nz;
    const int X0 = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int dj = threadIdx.y & 1, row = threadIdx.y >> 1;
    const int cy = blockIdx.y * kRestrictRows + row;
    const int cz0 = (int)blockIdx.z * czc;
    const int cz1 = cz0 + czc < cnz ? cz0 + czc : cnz;
    const bool row_on = cy < cny;
    const bool lane_on = X0 < cnx && row_on;
    const int iq = X0 < cnx ? X0 : 0;
    const int y = 2 * (row_on ? cy : 0) + dj;  // (rows past the end march a valid row; nothing is stored)
    const float* eo = e + half;  // black
    int ym, yp, il, ir;
    if (!wrap_axis(y - 1, ny, L.per[1], ym)) ym = y;
    if (!wrap_axis(y + 1, ny, L.per[1], yp)) yp = y;
    if (!wrap_axis(iq - 1, nxh, L.per[0], il)) il = iq;
    if (!wrap_axis(iq + 4, nxh, L.per[0], ir)) ir = iq;
    // row offsets carried from plane to plane (compact rows; natural: the
    // state bytes); z + 1 past the last plane is the first (periodic) or the
    // row itself (a wall)
    const int z0 = 2 * cz0, z1 = 2 * cz1;
    const int plane = nxh * ny, back = (nz - 1) * plane, zwall = L.per[2] ? 0 : 1;
    int orh = nxh * (y + ny * z0) + iq, oym = nxh * (ym + ny * z0) + iq, oyp = nxh * (yp + ny * z0) + iq;
    int ost = L.nx * (y + ny * z0) + 2 * iq;
    const int dl = il - iq, dr = ir - iq;
    // plane z's loads: the black rows (y, z+1), (y-1, z), (y+1, z), the halo
    // of (y, z), the red e and rhs of (y, z), the state bytes
    float F[4], A[4], B[4], Cr[4], R[4], h;
    uint2 sw;
    auto load = [&](int z, int rh, int hm, int hp, int so, float (&f)[4], float (&a)[4], float (&b)[4],
                    float (&c)[4], float (&r)[4], float& hv, uint2& s) {
        ES_VLD(f, 0, eo + (z + 1 < nz ? rh + plane : (zwall ? rh : rh - back)));
        ES_VLD(a, 0, eo + hm);
        ES_VLD(b, 0, eo + hp);
        ES_VLD(c, 0, e + rh);
        ES_VLD(r, 0, rhs + rh);
        hv = eo[rh + (((y + z) & 1) == 0 ? dl : dr)];
        s = *reinterpret_cast<const uint2*>(st + so);
    };
    float D[4], X[4];
    ES_VLD(D, 0, eo + (z0 > 0 ? orh - plane : (zwall ? orh : orh + back)));
    ES_VLD(X, 0, eo + orh);
    if (z0 < z1) load(z0, orh, oym, oyp, ost, F, A, B, Cr, R, h, sw);
    for (int z = z0; z < z1; z++) {
        float nF[4], nA[4], nB[4], nC[4], nR[4], nh = 0.0f;
        uint2 nsw = make_uint2(0u, 0u);
        if (z + 1 < z1)
            load(z + 1, orh + plane, oym + plane, oyp + plane, ost + L.nx * ny, nF, nA, nB, nC, nR, nh, nsw);
        const int O = (y + z) & 1;  // red cells of this row: x = 2 i + O
        const int rown = ost;
        // the black row with its halo: ox[0] left of X0 (O = 0), ox[5] right of X0+3 (O = 1)
        const float ox[6] = {O == 0 ? h : 0.0f, X[0], X[1], X[2], X[3], O == 1 ? h : 0.0f};
        float res[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int bit = 2 * k + O;
            const unsigned sv = ((bit < 4 ? sw.x : sw.y) >> (8 * (bit & 3))) & 0xFFu;
            res[k] = 0.0f;
            if ((sv & ST_KIND) != ST_UNKNOWN) continue;
            if (sv & ST_NEAR) {
                res[k] = near_res[rown + bit];
                continue;
            }
            float o = O == 0 ? ox[k] : ox[k + 1];  // (left, right, y-, y+, z-, z+ as k_restrict_v)
            o += O == 0 ? ox[k + 1] : ox[k + 2];
            o += A[k];
            o += B[k];
            o += D[k];
            o += F[k];
            res[k] = R[k] - (L.diag0 * Cr[k] - o) * inv_h2;
        }
        const int dk = z & 1, par = (z >> 1) & 1;
        part[par][row][2 * dk + dj][threadIdx.x] = make_float4(res[0], res[1], res[2], res[3]);
        if (dk == 1) {
            // (both warps of every row reach this together: whole planes, same bounds)
            __syncthreads();
            if (dj == 0 && lane_on) {
                // per fine row k_restrict_v adds (even child + odd child), one
                // of them the black child (0): the red residual plus 0
                float sum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float4 p = part[par][row][q][threadIdx.x];
                    sum[0] += p.x;
                    sum[1] += p.y;
                    sum[2] += p.z;
                    sum[3] += p.w;
                }
                const int cz = z >> 1;
                const int C = X0 + cnx * (cy + cny * cz);
                const uchar4 cs = *reinterpret_cast<const uchar4*>(cst + C);
                const uint8_t ck[4] = {cs.x, cs.y, cs.z, cs.w};
                float v[4];
#pragma unroll
                for (int k = 0; k < 4; k++) v[k] = ((ck[k] & ST_KIND) == ST_UNKNOWN) ? sum[k] / 8.0f : 0.0f;
                store_coarse4(crhs, C, (X0 + cy + cz) & 1, chalf, v);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            D[k] = X[k];
            X[k] = F[k];
            F[k] = nF[k];
            A[k] = nA[k];
            B[k] = nB[k];
            Cr[k] = nC[k];
            R[k] = nR[k];
        }
        h = nh;
        sw = nsw;
        orh += plane;
        oym += plane;
        oyp += plane;
        ost += L.nx * ny;
    }
}

// Coarsest level: one thread block holds the level in shared memory and
// runs `sweeps` red-black sweeps from a zero iterate.
template <class T>
__global__ void __launch_bounds__(1024) k_coarse_solve(Level<T> L, const uint8_t* st, const T* rhs, T* e,
                                                       int sweeps, T omega) {
    pdl_wait();
    extern __shared__ unsigned char smem[];
    const int n = L.nx * L.ny * L.nz;
    T* se = (T*)smem;
    T* sr = se + n;
    uint8_t* ss = (uint8_t*)(sr + n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        se[i] = (T)0;
        sr[i] = rhs[i];
        ss[i] = st[i];
    }
    __syncthreads();
    for (int s = 0; s < sweeps; s++)
        for (int colour = 0; colour < 2; colour++) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int x = i % L.nx, y = (i / L.nx) % L.ny, z = i / (L.nx * L.ny);
                if (((x + y + z) & 1) != colour) continue;
                const uint8_t k = ss[i];
                if ((k & ST_KIND) != ST_UNKNOWN) continue;
                T diag, off;
                level_stencil<T>(L, ss, se, x, y, z, k, diag, off);
                const T gs = (L.h2 * sr[i] + off) / diag;
                se[i] = ((T)1 - omega) * se[i] + omega * gs;
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) e[i] = se[i];
}

// Coarsest level, one block, from shared memory, with the unknown cells of
// each colour packed into a list: every lane of a half sweep updates a cell
// of that colour, so no lane idles on the other colour or past a short row
// (the FP64 form is bound by one SM's FP64 pipe here).  Set-up, once per
// launch: for each unknown cell a 4-byte record (x, y, z and a mask of its
// unknown neighbours) goes to its colour's list (shared-memory atomics; the
// order within a colour does not matter, its cells depend only on the other
// colour), and its inverse diagonal comes from a table of 1 / (diag0 + k),
// k = #Dirichlet - #Neumann faces (Sec. 5.4, as in level_stencil).  A sweep
// then needs no index division, no state lookup and no division.  A masked
// neighbour adds +0, so the sum is taken in level_stencil's order.
// Records hold coordinates in 8 bits: nx, ny, nz <= 256.
template <class T>
__global__ void __launch_bounds__(1024) k_coarse_lists(Level<T> L, const uint8_t* __restrict__ st,
                                                       const T* __restrict__ rhs, T* __restrict__ e, int sweeps,
                                                       T omega) {
    pdl_wait();
    extern __shared__ unsigned char smem[];
    __shared__ T inv_tab[13];  // 1 / (diag0 + k), k = -6 .. 6
    __shared__ int cnt[2];
    const int nx = L.nx, ny = L.ny, nz = L.nz, nxy = nx * ny, n = nxy * nz;
    T* se = (T*)smem;
    T* sr = se + n;
    T* sinv = sr + n;
    unsigned* rec = (unsigned*)(sinv + n);  // colour 0 from the front, colour 1 from the back
    if (threadIdx.x < 13) inv_tab[threadIdx.x] = (T)1 / (L.diag0 + (T)((int)threadIdx.x - 6));
    if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int x = i % nx, y = (i / nx) % ny, z = i / nxy;
        const uint8_t k = st[i];
        se[i] = (T)0;
        sr[i] = rhs[i];
        T inv = (T)0;
        if ((k & ST_KIND) == ST_UNKNOWN) {
            int dk = 0;
            unsigned m = 0;
            const int v[3] = {x, y, z}, n3[3] = {nx, ny, nz}, stride[3] = {1, nx, nxy};
            for (int a = 0; a < 3; a++)
                for (int sd = 0; sd < 2; sd++) {
                    int p = v[a] + (sd ? 1 : -1);
                    if (p < 0 || p >= n3[a]) {
                        if (!L.per[a]) {
                            dk += L.pot_bc[2 * a + sd] == ES_POT_DIRICHLET ? 1 : -1;
                            continue;
                        }
                        p = p < 0 ? p + n3[a] : p - n3[a];
                    }
                    const uint8_t kn = st[i + (p - v[a]) * stride[a]] & ST_KIND;
                    if (kn == ST_UNKNOWN)
                        m |= 1u << (2 * a + sd);
                    else
                        dk += kn == ST_DIR ? 1 : -1;
                }
            inv = inv_tab[dk + 6];
            const int col = (x + y + z) & 1;
            const int pos = atomicAdd(&cnt[col], 1);
            rec[col == 0 ? pos : n - 1 - pos] = (unsigned)x | ((unsigned)y << 8) | ((unsigned)z << 16) | (m << 24);
        }
        sinv[i] = inv;
    }
    __syncthreads();
    const int c0 = cnt[0], c1 = cnt[1];
    for (int s = 0; s < sweeps; s++)
        for (int colour = 0; colour < 2; colour++) {
            const int m_ = colour == 0 ? c0 : c1;
            for (int j = threadIdx.x; j < m_; j += blockDim.x) {
                const unsigned r = rec[colour == 0 ? j : n - 1 - j];
                const int x = r & 0xFF, y = (r >> 8) & 0xFF, z = (r >> 16) & 0xFF;
                const unsigned m = r >> 24;
                const int i = x + nx * y + nxy * z;
                const int xm = x == 0 ? nx - 1 : -1, xp = x == nx - 1 ? 1 - nx : 1;
                const int ym = y == 0 ? (ny - 1) * nx : -nx, yp = y == ny - 1 ? (1 - ny) * nx : nx;
                const int zm = z == 0 ? (nz - 1) * nxy : -nxy, zp = z == nz - 1 ? (1 - nz) * nxy : nxy;
                T o = (T)0;
                o += (m & 1) ? se[i + xm] : (T)0;
                o += (m & 2) ? se[i + xp] : (T)0;
                o += (m & 4) ? se[i + ym] : (T)0;
                o += (m & 8) ? se[i + yp] : (T)0;
                o += (m & 16) ? se[i + zm] : (T)0;
                o += (m & 32) ? se[i + zp] : (T)0;
                const T gs = (L.h2 * sr[i] + o) * sinv[i];
                se[i] = ((T)1 - omega) * se[i] + omega * gs;
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) e[i] = se[i];
}

template <class T>
__global__ void k_zero(T* p, int n) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (T)0;
}

// psi += e at unknown cells (FP64 form).
__global__ void k_correct(int N, const uint8_t* __restrict__ st0, const double* __restrict__ e,
                          double* __restrict__ psi) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    if ((st0[c] & ST_KIND) != ST_UNKNOWN) return;
    psi[c] += e[c];
}

// psi += e at unknown cells, psi in float-float (MIXED32 form); four cells
// per thread with 16-byte accesses, the last thread also takes the N % 4
// tail cells one by one.
// SPLIT: e in the colour-split layout (nx % 8 == 0, so N % 4 == 0 and a
// 4-cell group never wraps a row; its colour follows from its position).
template <class E, bool SPLIT = false>
__global__ void k_correct_ff(int N, const uint8_t* __restrict__ st0, const E* __restrict__ e,
                             float* __restrict__ psi_hi, float* __restrict__ psi_lo, EAcc<float, E> A,
                             int nx = 0, int ny = 0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int N4 = N >> 2;
    if (i == N4 - 1 || (N4 == 0 && i == 0))
        for (int c = 4 * N4; c < N; c++)
            if ((st0[c] & ST_KIND) == ST_UNKNOWN) {
                const ff v = ff_add_f({psi_hi[c], psi_lo[c]}, A.ld(e + c));
                psi_hi[c] = v.hi;
                psi_lo[c] = v.lo;
            }
    if (i >= N4) return;
    const uchar4 st = reinterpret_cast<const uchar4*>(st0)[i];
    Q4<float> ev;
    if constexpr (SPLIT) {
        const int c = 4 * i, row = c / nx;  // (row = y + ny z)
        ev = rb_ld4(e, N >> 1, c, (c - row * nx + row % ny + row / ny) & 1);
    } else {
        ev = A.ld4(e + 4 * (size_t)i);
    }
    float4 h = reinterpret_cast<float4*>(psi_hi)[i], l = reinterpret_cast<float4*>(psi_lo)[i];
    const uint8_t sv[4] = {st.x, st.y, st.z, st.w};
    const float evv[4] = {ev.v0, ev.v1, ev.v2, ev.v3};
    float hv[4] = {h.x, h.y, h.z, h.w}, lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if ((sv[k] & ST_KIND) != ST_UNKNOWN) continue;
        const ff v = ff_add_f({hv[k], lv[k]}, evv[k]);
        hv[k] = v.hi;
        lv[k] = v.lo;
    }
    reinterpret_cast<float4*>(psi_hi)[i] = make_float4(hv[0], hv[1], hv[2], hv[3]);
    reinterpret_cast<float4*>(psi_lo)[i] = make_float4(lv[0], lv[1], lv[2], lv[3]);
}

// MIXED32: psi (float-float) from doubles, and back.
__global__ void k_split_psi(int N, const double* __restrict__ src, float* __restrict__ hi, float* __restrict__ lo) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const ff v = ff_from_double(src[c]);
    hi[c] = v.hi;
    lo[c] = v.lo;
}

__global__ void k_join_psi(int N, const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ dst) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) dst[c] = (double)hi[c] + (double)lo[c];
}

// --- EDL field and body force (Sec. 5.6) ---

// Value across face (a, side) of unknown cell c for a D3Q7 central
// difference: neighbour value, or the boundary value extrapolated from the
// cell (Dirichlet: 2 v - psi_c; Neumann: psi_c + sigma/eps; wall: psi_c).
template <class P>
__device__ __forceinline__ P face_value(const Grid& g, const Solver& s, const P* psi, const int32_t* owner,
                                        const DParticle* part, const int* kind, int x, int y, int z, P pc, int a,
                                        int side) {
    int d[3] = {0, 0, 0};
    d[a] = side;
    long long nb;
    if (!neighbour(g, x, y, z, d[0], d[1], d[2], nb)) {
        int face = 2 * a + (side > 0 ? 1 : 0);
        return s.pot_bc[face] == ES_POT_DIRICHLET ? (P)(2.0 * s.pot_val[face]) - pc : pc;
    }
    int o = owner[nb];
    if (o < 0) return psi[nb];
    if (kind[o] == ES_KIND_ZETA) return (P)(2.0 * part[o].zeta) - pc;
    return pc + (P)(part[o].sigma / s.eps);
}

// The same ghost values in FP32 for the reduced forms: the sphere's
// boundary value (2 zeta or sigma / eps) comes from its float-float record
// (high part), a Dirichlet wall's 2 * value from wall2.
struct WallF {
    float v2[6];
};
__device__ __forceinline__ float face_value_f(const Grid& g, const Solver& s, const WallF& wall2,
                                              const float* psi, const int32_t* owner, const uint8_t* st0,
                                              const float2* pbc, int x, int y, int z, float pc, int a, int side) {
    int d[3] = {0, 0, 0};
    d[a] = side;
    long long nb;
    if (!neighbour(g, x, y, z, d[0], d[1], d[2], nb)) {
        const int face = 2 * a + (side > 0 ? 1 : 0);
        return s.pot_bc[face] == ES_POT_DIRICHLET ? wall2.v2[face] - pc : pc;
    }
    const uint8_t k = st0[nb] & ST_KIND;
    if (k == ST_UNKNOWN) return psi[nb];
    const float b = pbc[owner[nb]].x;
    return k == ST_DIR ? b - pc : pc + b;
}

// f_b = rho_e (E_ext - grad psi), rho_e = -kappa^2 eps psi (Eq. ChrgDensDHA),
// computed in the type P of the potential it reads (double, or the float
// high part of psi in the reduced forms) and stored in the type S of f_b.
template <class S, class P>
__global__ void __launch_bounds__(128) k_body_force(Grid g, Solver s, P Ex, P Ey, P Ez, P k2e, P phi_t,
                                                    const P* __restrict__ psi, const uint8_t* __restrict__ flags,
                                                    const int32_t* __restrict__ owner,
                                                    const DParticle* __restrict__ part, const int* __restrict__ kind,
                                                    const uint8_t* __restrict__ st0, const float2* __restrict__ pbc,
                                                    WallF wall2, S* __restrict__ fb) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int nx = g.nx, nxy = g.nx * g.ny;
    const int c = x + nx * (y + g.ny * z);
    const uint8_t fl = flags[c];
    P f0 = (P)0, f1 = (P)0, f2 = (P)0;
    if (!(fl & F_SOLID)) {
        const P pc = psi[c];
        P g0, g1, g2;
        if (!(fl & F_NEAR19)) {
            // isotropic D3Q19 gradient (1/c_s^2) sum_q w_q psi(x + e_q) e_q,
            // taken pairwise: 3 w_q (psi(x + e_q) - psi(x - e_q)) e_q
            const int dx[3] = {(x == 0 ? nx - 1 : x - 1) - x, 0, (x == nx - 1 ? 0 : x + 1) - x};
            const int dy[3] = {((y == 0 ? g.ny - 1 : y - 1) - y) * nx, 0, ((y == g.ny - 1 ? 0 : y + 1) - y) * nx};
            const int dz[3] = {((z == 0 ? g.nz - 1 : z - 1) - z) * nxy, 0, ((z == g.nz - 1 ? 0 : z + 1) - z) * nxy};
            g0 = (P)0;
            g1 = (P)0;
            g2 = (P)0;
#pragma unroll
            for (int q = 1; q <= 9; q++) {
                const int op = dx[1 + cx(q)] + dy[1 + cy(q)] + dz[1 + cz(q)];
                const int om = dx[1 - cx(q)] + dy[1 - cy(q)] + dz[1 - cz(q)];
                const P d = (P)(3.0 * wq(q)) * (psi[c + op] - psi[c + om]);
                if (cx(q)) g0 += cx(q) > 0 ? d : -d;
                if (cy(q)) g1 += cy(q) > 0 ? d : -d;
                if (cz(q)) g2 += cz(q) > 0 ? d : -d;
            }
        } else if constexpr (sizeof(P) == 4) {
            g0 = 0.5f * (face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 0, 1) -
                         face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 0, -1));
            g1 = 0.5f * (face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 1, 1) -
                         face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 1, -1));
            g2 = 0.5f * (face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 2, 1) -
                         face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 2, -1));
        } else {
            g0 = (P)0.5 * (face_value<P>(g, s, psi, owner, part, kind, x, y, z, pc, 0, 1) -
                           face_value<P>(g, s, psi, owner, part, kind, x, y, z, pc, 0, -1));
            g1 = (P)0.5 * (face_value<P>(g, s, psi, owner, part, kind, x, y, z, pc, 1, 1) -
                           face_value<P>(g, s, psi, owner, part, kind, x, y, z, pc, 1, -1));
            g2 = (P)0.5 * (face_value<P>(g, s, psi, owner, part, kind, x, y, z, pc, 2, 1) -
                           face_value<P>(g, s, psi, owner, part, kind, x, y, z, pc, 2, -1));
        }
        // (phi_t > 0: the nonlinear Poisson-Boltzmann charge density)
        const P rho_e = phi_t > (P)0 ? -k2e * phi_t * sinh(pc / phi_t) : -k2e * pc;
        f0 = rho_e * (Ex - g0);
        f1 = rho_e * (Ey - g1);
        f2 = rho_e * (Ez - g2);
    }
    fb[c] = (S)f0;
    fb[(long long)g.N + c] = (S)f1;
    fb[2LL * g.N + c] = (S)f2;
}

// Body force of the reduced forms, 4-cell spans (16-byte loads of the nine
// rows the D3Q19 gradient touches).  Interior fluid cells take the
// isotropic gradient (Eq. ElPotGradComp, pairwise as in k_body_force);
// obstacle cells get 0; cells with a non-fluid D3Q19 neighbour are written
// again right after by k_body_force_near with the D3Q7 ghost-value gradient.
__global__ void __launch_bounds__(256) k_body_force_v(Grid g, float Ex, float Ey, float Ez, float k2e,
                                                      const float* __restrict__ psi,
                                                      const uint8_t* __restrict__ flags, float* __restrict__ fb) {
    const int xs = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
    if (xs >= g.nx || y >= g.ny) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    // periodic wrap; beyond a wall the cells are near cells (rewritten), so
    // any valid index does
    const int xl = xs == 0 ? (g.per[0] ? nx - 1 : 0) : xs - 1;
    const int xr = xs + 4 == nx ? (g.per[0] ? 0 : nx - 1) : xs + 4;
    const int ym = y == 0 ? (g.per[1] ? ny - 1 : 0) : y - 1, yp = y == ny - 1 ? (g.per[1] ? 0 : y) : y + 1;
    const int zm = z == 0 ? (g.per[2] ? nz - 1 : 0) : z - 1, zp = z == nz - 1 ? (g.per[2] ? 0 : z) : z + 1;
    auto rowp = [&](int yy, int zz) { return psi + nx * (yy + ny * zz); };
    auto span6 = [&](const float* r, float (&v)[6]) {
        const float4 q = *reinterpret_cast<const float4*>(r + xs);
        v[0] = r[xl];
        v[1] = q.x;
        v[2] = q.y;
        v[3] = q.z;
        v[4] = q.w;
        v[5] = r[xr];
    };
    auto span4 = [&](const float* r, float (&v)[4]) {
        const float4 q = *reinterpret_cast<const float4*>(r + xs);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    };
    float c0[6], ym0[6], yp0[6], zm0[6], zp0[6], mm[4], pm[4], mp[4], pp[4];
    span6(rowp(y, z), c0);
    span6(rowp(ym, z), ym0);
    span6(rowp(yp, z), yp0);
    span6(rowp(y, zm), zm0);
    span6(rowp(y, zp), zp0);
    span4(rowp(ym, zm), mm);  // (y-1, z-1)
    span4(rowp(yp, zm), pm);  // (y+1, z-1)
    span4(rowp(ym, zp), mp);  // (y-1, z+1)
    span4(rowp(yp, zp), pp);  // (y+1, z+1)
    const int row = nx * (y + ny * z);
    const uchar4 f4 = *reinterpret_cast<const uchar4*>(flags + row + xs);
    const uint8_t fl[4] = {f4.x, f4.y, f4.z, f4.w};
    float o0[4], o1[4], o2[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int j = i + 1;  // index in the 6-wide rows
        const Psi19 p{c0[j],      c0[j + 1],  c0[j - 1],  yp0[j],     ym0[j],     zp0[j],     zm0[j],
                      yp0[j + 1], ym0[j - 1], ym0[j + 1], yp0[j - 1], zp0[j + 1], zm0[j - 1], zm0[j + 1],
                      zp0[j - 1], pp[i],      mm[i],      pm[i],      mp[i]};
        float f0, f1, f2;
        body_force_iso(p, Ex, Ey, Ez, k2e, f0, f1, f2);
        const bool solid = fl[i] & F_SOLID;
        o0[i] = solid ? 0.0f : f0;
        o1[i] = solid ? 0.0f : f1;
        o2[i] = solid ? 0.0f : f2;
    }
    const size_t N = (size_t)g.N;
    *reinterpret_cast<float4*>(fb + row + xs) = make_float4(o0[0], o0[1], o0[2], o0[3]);
    *reinterpret_cast<float4*>(fb + N + row + xs) = make_float4(o1[0], o1[1], o1[2], o1[3]);
    *reinterpret_cast<float4*>(fb + 2 * N + row + xs) = make_float4(o2[0], o2[1], o2[2], o2[3]);
}

// The fluid cells with a non-fluid D3Q19 neighbour: D3Q7 gradient with the
// ghost values of face_value_f (list of cells, kNearSegs segments).
__global__ void __launch_bounds__(256) k_body_force_near(Grid g, Solver s, float Ex, float Ey, float Ez, float k2e,
                                                         const float* __restrict__ psi,
                                                         const int32_t* __restrict__ owner,
                                                         const uint8_t* __restrict__ st0,
                                                         const float2* __restrict__ pbc, WallF wall2,
                                                         const int* __restrict__ list,
                                                         const int* __restrict__ count, int cap,
                                                         float* __restrict__ fb) {
    const int n = count[blockIdx.y];
    const int* seg = list + (size_t)blockIdx.y * cap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = seg[i];
        const int x = c % g.nx, yz = c / g.nx, y = yz % g.ny, z = yz / g.ny;
        const float pc = psi[c];
        const float g0 = 0.5f * (face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 0, 1) -
                                 face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 0, -1));
        const float g1 = 0.5f * (face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 1, 1) -
                                 face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 1, -1));
        const float g2 = 0.5f * (face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 2, 1) -
                                 face_value_f(g, s, wall2, psi, owner, st0, pbc, x, y, z, pc, 2, -1));
        const float rho_e = -k2e * pc;
        fb[c] = rho_e * (Ex - g0);
        fb[(size_t)g.N + c] = rho_e * (Ey - g1);
        fb[2 * (size_t)g.N + c] = rho_e * (Ez - g2);
    }
}

template <class T>
Level<T> level_desc(const es_ctx* c, int l) {
    Level<T> L;
    L.nx = c->ln[l][0];
    L.ny = c->ln[l][1];
    L.nz = c->ln[l][2];
    for (int a = 0; a < 3; a++) L.per[a] = c->g.per[a];
    for (int f = 0; f < 6; f++) L.pot_bc[f] = c->S.pot_bc[f];
    double h = (double)(1 << l);
    L.h2 = (T)(h * h);
    L.diag0 = (T)(6.0 + c->S.kappa * c->S.kappa * h * h);
    return L;
}

// Shared memory of the staged finest-level half sweep (0: not staged).
size_t bulk_smem_bytes(const es_ctx* c) {
    const int nxh = c->ln[0][0] / 2;
    if (!c->rb0 || nxh > 256 || c->P.sweep_staging != ES_STAGE_BULK) return 0;
    const int ty = 256 / (nxh / 4);
    return (size_t)kBulkSlots * (2 * ty + 2) * nxh * sizeof(float);
}

// The coarsest level runs in one block from shared memory: from packed
// per-colour lists (k_coarse_lists: e, rhs, inverse diagonal, one 4-byte
// record per cell) when that fits, else k_coarse_solve (e, rhs, states).
size_t coarse_cells(const es_ctx* c) { return (size_t)c->ln[c->L - 1][0] * c->ln[c->L - 1][1] * c->ln[c->L - 1][2]; }

bool coarse_by_lists(const es_ctx* c, size_t tsize) {
    const int* m = c->ln[c->L - 1];
    return m[0] <= 256 && m[1] <= 256 && m[2] <= 256 && coarse_cells(c) * (3 * tsize + 4) <= 200 * 1024;
}

size_t coarse_smem_bytes(const es_ctx* c, size_t tsize) {
    const size_t n = coarse_cells(c);
    return coarse_by_lists(c, tsize) ? n * (3 * tsize + 4) : n * (2 * tsize + 1);
}

// Levels up to this many cells (near_list_cells, default 2^21) update their
// near-boundary cells inside the smoothing kernel; larger ones in a separate
// pass over the near-cell list.
long long inline_near_cells(const es_ctx* c) {
    return c->P.near_list_cells > 0 ? (long long)c->P.near_list_cells : (long long)ES_NEAR_LIST_CELLS;
}

// Launch shape of the fused sweep: 128 x 12 output tiles, and the z extent
// cut into chunks so that the blocks fill whole waves of the resident-block
// capacity; a chunk re-reads three planes and recomputes two red planes, so
// the cost model is (waves rounded up) x (chunk + 2).
template <class T>
dim3 rb_launch_shape(es_ctx* c, const Level<T>& L, int& zc) {
    const int ti = sizeof(T) == 4 ? 0 : 1;
    if (c->rb_blocks[ti] == 0) {
        cudaFuncSetAttribute(k_smooth_rb2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RB2<T>::smem);
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_smooth_rb2<T>, 32 * (kRbRows + 1), RB2<T>::smem) !=
                cudaSuccess ||
            b < 1) {
            cudaGetLastError();
            b = 1;
        }
        c->rb_blocks[ti] = b;
    }
    const long long cols = (long long)(L.nx / 128) * ((L.ny + kRbOut - 1) / kRbOut);
    const long long cap = (long long)c->rb_blocks[ti] * c->n_sm;
    double best = 1e300;
    int best_zc = L.nz;
    for (int chunks = 1; chunks <= L.nz && chunks <= 64; chunks++) {
        const int z = (L.nz + chunks - 1) / chunks;
        const long long nb = cols * ((L.nz + z - 1) / z);
        const double waves = (double)((nb + cap - 1) / cap);
        const double cost = waves * (z + 2);
        if (cost < best - 1e-9) {
            best = cost;
            best_zc = z;
        }
    }
    zc = best_zc;
    return dim3((unsigned)(L.nx / 128), (unsigned)((L.ny + kRbOut - 1) / kRbOut), (unsigned)((L.nz + zc - 1) / zc));
}

// One V-cycle on level l for A e = rhs (the result in e[l]).  warm != 0
// (level 0 only): the current iterate is improved instead of starting from
// zero.  Algorithmic bytes of each launch (for es_profile): a fused sweep
// reads e, rhs and the state byte and writes e once per cell (e is not read
// on a zero start); a half sweep reads e and the states of all cells and
// rhs of half of them and writes half of e (all of e on a zero start);
// restriction and prolongation read the fine e and rhs (or e twice) and
// states and touch the coarse level once.
template <class T>
cudaError_t vcycle_level(es_ctx* c, int l, int warm);

// One level of the V-cycle with the level's correction stored as E (T, or
// FP16 on the finest level under ES_MG_FP16: two-pass vector smoother,
// never the coarsest level; the parameters are checked at creation).
template <class T, class E>
cudaError_t vcycle_impl(es_ctx* c, int l, int warm) {
    constexpr bool kNative = std::is_same<T, E>::value;
    Level<T> L = level_desc<T>(c, l);
    E* e = (E*)c->e[l];
    T* rhs = (T*)c->rhs[l];
    const uint8_t* st = c->st[l];
    const T omega = (T)c->P.omega;
    const T inv_diag0 = (T)1 / L.diag0;
    const int Nl = L.nx * L.ny * L.nz;
    EAcc<T, E> A{(T)1, (T)1};
    if constexpr (!kNative) A = EAcc<T, E>{(T)c->e_scale, (T)1 / (T)c->e_scale};
    dim3 blk(128);
    dim3 half(((L.nx + 1) / 2 + 127) / 128, L.ny, L.nz);
    dim3 full((L.nx + 127) / 128, L.ny, L.nz);
    const bool vec = (L.nx % 4) == 0;
    constexpr int W = 4;
    dim3 vblk(32, 8), vgrd((L.nx / W + 31) / 32, (L.ny + 7) / 8, L.nz);

    // (the span form needs whole 128-cell tiles in x; a periodic axis of
    // one cell is its own neighbour: no red-black split)
    const bool use_rb = kNative && c->P.smoother == ES_SMOOTH_FUSED && (L.nx % 128) == 0 &&
                        (!L.per[1] || L.ny >= 2) && (!L.per[2] || L.nz >= 2);
    // levels of the reduced forms in the colour-split layout (the finest,
    // and level 1 when it is split as well)
    const bool split = kNative && std::is_same<T, float>::value && split_level(c, l);
    const uint32_t* rbmask = l == 0 ? c->rbmask : c->rbmask1;
    const int rb_wpr = l == 0 ? c->rb_wpr : c->rb_wpr1;
    // half the cells of the next level when it is split too (its right-hand
    // side is restricted, and its correction prolonged, in that layout)
    const int chalf = split && l + 1 < c->L && split_level(c, l + 1)
                          ? c->ln[l + 1][0] * c->ln[l + 1][1] * c->ln[l + 1][2] / 2
                          : 0;
    const RbMap rb{Nl / 2};
    // reduced forms, Gauss-Seidel: the pre-smoothing ends with a black half
    // sweep, after which only red residuals remain (the restriction adds the
    // red children only; the same in both finest-level layouts)
    const bool red_only = kNative && std::is_same<T, float>::value && c->P.omega == 1.0 && c->P.nu1 >= 1;
    int rb_zc = 1;
    dim3 rb_grid(1, 1, 1);
    if (use_rb) rb_grid = rb_launch_shape<T>(c, L, rb_zc);
    const double nl = (double)Nl, ts = (double)sizeof(T), es = (double)sizeof(E);
    const int* mc = l + 1 < c->L ? c->ln[l + 1] : c->ln[l];
    const double nc = (double)mc[0] * mc[1] * mc[2];
    auto sweep = [&](int first) {
        if constexpr (kNative) {
            if (use_rb) {
                ProfScope ps(c, "smooth_fused", l, nl * ((first ? 2.0 : 3.0) * ts + 1.0));
                T* eo = (T*)c->e2[l];
                launch_pdl(c, k_smooth_rb2<T>, rb_grid, dim3(32, kRbRows + 1), RB2<T>::smem, L, inv_diag0, st, rhs, e,
                           eo, first, omega, rb_zc);
                c->e2[l] = c->e[l];
                c->e[l] = eo;
                e = eo;
                count(c);
                return;
            }
        }
        // per half sweep: e of every cell in, the colour's e out, its rhs
        // and state bytes in
        const double b_first = nl * (0.5 * es + 0.5 * ts + 1.0), b_half = nl * (1.5 * es + 0.5 * ts + 1.0);
        if constexpr (kNative && std::is_same<T, float>::value) {
            if (split) {
                // colour-split finest level: interior pass, then the colour's
                // near-boundary cells from the list
                // planes per block: up to 16, keeping about eight blocks per
                // SM in all
                const int gx = (L.nx / 8 + 31) / 32, gy = (L.ny + 7) / 8;
                int zc = (int)((long long)gx * gy * L.nz / (8LL * c->n_sm));
                zc = zc < 1 ? 1 : (zc > 16 ? 16 : zc);
                const dim3 sgrd(gx, gy, (L.nz + zc - 1) / zc);
                const int* cnt = c->near_count + 2 * kNearSegs * l;
                // per cell: the other colour's e in, the colour's e out, its
                // rhs in (from zero: rhs in, e out), the mask bits; the
                // colour's old e in as well unless omega = 1 (the
                // near-boundary cells' scattered loads are not counted)
                const double own = c->P.omega == 1.0 ? 0.0 : 0.5 * es;
                const double b_rb_first = nl * (0.5 * es + 0.5 * ts + 0.0625);
                const double b_rb_half = nl * (1.0 * es + own + 0.5 * ts + 0.0625);
                const NearWork nw{st, c->near_list[l], cnt, c->near_cap[l]};
                // rows of up to 256 compact cells: staged by bulk copies on request
                const int nxh = L.nx / 2;
                const bool bulk = l == 0 && nxh <= 256 && c->P.sweep_staging == ES_STAGE_BULK;
                BulkShape bs{nxh / 4, 0, 0};
                dim3 bgrd;
                size_t bsm = 0;
                if (bulk) {
                    bs.ty = 256 / bs.tpr;
                    const int ytiles = (L.ny + bs.ty - 1) / bs.ty;
                    bsm = bulk_smem_bytes(c);
                    // planes per block: the grid should fill whole waves of
                    // the resident blocks, and each block pays two planes of
                    // pipeline start-up; cost ~ waves x (planes + 2)
                    const long long cap = (long long)(c->bulk_blocks > 0 ? c->bulk_blocks : 1) * c->n_sm;
                    double best = 1e300;
                    for (int zq = 4; zq <= 32 && zq <= L.nz; zq++) {
                        const long long nb = (long long)ytiles * ((L.nz + zq - 1) / zq);
                        const double cost = (double)((nb + cap - 1) / cap) * (zq + 2);
                        if (cost < best - 1e-9) {
                            best = cost;
                            bs.zc = zq;
                        }
                    }
                    if (bs.zc == 0) bs.zc = L.nz;
                    bgrd = dim3(ytiles, (L.nz + bs.zc - 1) / bs.zc);
                }
                for (int col = 0; col < 2; col++) {
                    const int fs = first ? (col == 0 ? 1 : 2) : 0;
                    ProfScope ps(c, "smooth_half", l,
                                 !first ? b_rb_half : (col == 0 ? b_rb_first : b_rb_half - nl * own));
                    if (bulk)
                        launch_pdl(c, k_smooth_rb_bulk<T>, bgrd, 256, bsm, L, inv_diag0, rbmask, rb_wpr, rhs, e, col,
                                   fs, omega, rb.half, nw, bs, c->d_status);
                    else
                        launch_pdl(c, k_smooth_rb<T>, sgrd, vblk, 0, L, inv_diag0, rbmask, rb_wpr, rhs, e, col, fs,
                                   omega, rb.half, nw, zc);
                }
                count(c, 2);
                return;
            }
        }
        if (vec) {
            const NearWork nwl{st, c->near_list[l], c->near_count + 2 * kNearSegs * l, c->near_cap[l]};
            if (Nl <= inline_near_cells(c)) {
                {
                    ProfScope ps(c, "smooth_half", l, first ? b_first : b_half);
                    launch_pdl(c, k_smooth_v<T, W, true, E>, vgrd, vblk, 0, L, inv_diag0, st, rhs, e, 0, first, omega,
                               A, nwl);
                }
                ProfScope ps(c, "smooth_half", l, b_half);
                launch_pdl(c, k_smooth_v<T, W, true, E>, vgrd, vblk, 0, L, inv_diag0, st, rhs, e, 1, 0, omega, A, nwl);
                count(c, 2);
                return;
            }
            // larger levels: the near-boundary cells from the list, in the
            // same launches (bytes: the spans' only; the list's scattered
            // loads are not counted)
            {
                ProfScope ps(c, "smooth_half", l, first ? b_first : b_half);
                launch_pdl(c, k_smooth_v<T, W, false, E>, vgrd, vblk, 0, L, inv_diag0, st, rhs, e, 0, first, omega, A,
                           nwl);
            }
            ProfScope ps(c, "smooth_half", l, b_half);
            launch_pdl(c, k_smooth_v<T, W, false, E>, vgrd, vblk, 0, L, inv_diag0, st, rhs, e, 1, 0, omega, A, nwl);
            count(c, 2);
            return;
        }
        if constexpr (kNative) {
            {
                ProfScope ps(c, "smooth_half", l, first ? b_first : b_half);
                launch_pdl(c, k_smooth<T>, half, blk, 0, L, st, rhs, e, 0, first, omega, (const T*)nullptr);
            }
            ProfScope ps(c, "smooth_half", l, b_half);
            launch_pdl(c, k_smooth<T>, half, blk, 0, L, st, rhs, e, 1, 0, omega, (const T*)nullptr);
            count(c, 2);
        }
    };
    if constexpr (kNative) {
        if (l == c->L - 1 && c->dk) {
            // nonlinear Poisson-Boltzmann (one level): red-black SOR sweeps on
            // the Newton system with the linearised centre entries
            for (int s = 0; s < c->P.coarse_sweeps; s++) {
                {
                    ProfScope ps(c, "smooth_half", l, nl * (2.0 * ts + 1.0));
                    launch_pdl(c, k_smooth<T>, half, blk, 0, L, st, rhs, e, 0, s == 0, omega, (const T*)c->dk);
                }
                ProfScope ps(c, "smooth_half", l, nl * (2.0 * ts + 1.0));
                launch_pdl(c, k_smooth<T>, half, blk, 0, L, st, rhs, e, 1, 0, omega, (const T*)c->dk);
                count(c, 2);
            }
            if (c->P.coarse_sweeps == 0) {
                cudaError_t err = cudaMemsetAsync(e, 0, (size_t)Nl * sizeof(T), c->stream);
                if (err != cudaSuccess) return err;
            }
            return cudaGetLastError();
        }
        if (l == c->L - 1) {
            size_t sm = coarse_smem_bytes(c, sizeof(T));
            if (sm <= 200 * 1024) {
                ProfScope ps(c, "coarse_solve", l, nl * (2.0 * ts + 1.0));
                if (coarse_by_lists(c, sizeof(T)))
                    launch_pdl(c, k_coarse_lists<T>, 1, 1024, sm, L, st, rhs, e, c->P.coarse_sweeps, omega);
                else
                    launch_pdl(c, k_coarse_solve<T>, 1, 1024, sm, L, st, rhs, e, c->P.coarse_sweeps, omega);
                count(c);
            } else {
                if (c->P.coarse_sweeps == 0) {
                    launch_pdl(c, k_zero<T>, (Nl + 255) / 256, 256, 0, e, Nl);
                    count(c);
                }
                for (int s = 0; s < c->P.coarse_sweeps; s++) sweep(s == 0);
            }
            return cudaGetLastError();
        }
    }
    const bool zero_start = !warm;
    if (c->P.nu1 == 0 && zero_start) {
        cudaError_t err = cudaMemsetAsync(e, 0, (size_t)Nl * sizeof(E), c->stream);  // (0 in every E)
        if (err != cudaSuccess) return err;
    }
    for (int s = 0; s < c->P.nu1; s++) sweep(s == 0 && zero_start);
    const int* m = c->ln[l + 1];
    const double b_grid = nl * (es + ts + 1.0) + nc * (ts + 1.0);
    {
        ProfScope ps_r(c, "restrict", l, b_grid);
        if (vec) {
            dim3 rgrd((m[0] / 2 + 31) / 32, (m[1] + 7) / 8, m[2]);
            T* scratch = (T*)c->e2[l];  // (the fused sweep's second iterate; free between sweeps)
            const dim3 ngrd(near_grid_x(c), 2 * kNearSegs);
            const int* cnt = c->near_count + 2 * kNearSegs * l;
            bool done = false;
            if constexpr (kNative && std::is_same<T, float>::value) {
                if (split && red_only) {
                    // (red near cells only: the first kNearSegs segments)
                    launch_pdl(c, k_near_residual<T, E, RbMap>, dim3(ngrd.x, kNearSegs), 256, 0, L, st, rhs, e,
                               c->near_list[l], cnt, c->near_cap[l], (T)1 / L.h2, scratch, A, rb);
                    // coarse planes per block: up to 8, about 16 blocks per SM in all
                    const int qx = (m[0] / 4 + 31) / 32, qy = (m[1] + kRestrictRows - 1) / kRestrictRows;
                    int czc = (int)((long long)qx * qy * m[2] / (16LL * c->n_sm));
                    czc = czc < 1 ? 1 : (czc > 8 ? 8 : czc);
                    const dim3 qgrd(qx, qy, (m[2] + czc - 1) / czc);
                    launch_pdl(c, k_restrict_red_rb, qgrd, dim3(32, 2 * kRestrictRows), 0, L, (T)1 / L.h2, st, rhs, e,
                               scratch, m[0], m[1], m[2], c->st[l + 1], (T*)c->rhs[l + 1], rb.half, chalf, czc);
                    done = true;
                } else if (split) {
                    launch_pdl(c, k_near_residual<T, E, RbMap>, ngrd, 256, 0, L, st, rhs, e, c->near_list[l], cnt,
                               c->near_cap[l], (T)1 / L.h2, scratch, A, rb);
                    const dim3 qgrd((m[0] / 4 + 31) / 32, (m[1] + 1) / 2, m[2]);
                    launch_pdl(c, k_restrict_rb, qgrd, vblk, 0, L, (T)1 / L.h2, st, rhs, e, scratch, m[0], m[1],
                               c->st[l + 1], (T*)c->rhs[l + 1], rb.half, chalf);
                    done = true;
                }
            }
            if (!done) {
                launch_pdl(c, k_near_residual<T, E>, ngrd, 256, 0, L, st, rhs, e, c->near_list[l], cnt, c->near_cap[l],
                           (T)1 / L.h2, scratch, A, NatMap{});
                launch_pdl(c, k_restrict_v<T, E>, rgrd, vblk, 0, L, inv_diag0, (T)1 / L.h2, st, rhs, e, scratch, m[0],
                           m[1], c->st[l + 1], (T*)c->rhs[l + 1], A, 0, red_only ? 1 : 0);
            }
            count(c, 2);
        } else if constexpr (kNative) {
            dim3 cgrid((m[0] + 127) / 128, m[1], m[2]);
            launch_pdl(c, k_residual_restrict<T>, cgrid, blk, 0, L, st, rhs, e, m[0], m[1], c->st[l + 1],
                       (T*)c->rhs[l + 1]);
            count(c);
        }
    }
    cudaError_t err = vcycle_level<T>(c, l + 1, 0);
    if (err != cudaSuccess) return err;
    {
        // (the black cells only ahead of a Gauss-Seidel post-smoothing: e in
        // and out for half the cells)
        const bool black_only = split && c->P.omega == 1.0 && c->P.nu2 >= 1;
        ProfScope ps(c, "prolong", l,
                     nl * ((black_only ? 1.0 : 2.0) * es + 1.0) + nc * (ts + 1.0));
        bool done = false;
        if constexpr (kNative && std::is_same<T, float>::value) {
            if (black_only) {
                const dim3 bgrd((L.nx / 8 + 31) / 32, (L.ny + 7) / 8, L.nz);
                launch_pdl(c, k_prolong_black_rb, bgrd, vblk, 0, L, st, e, rb.half, m[0], m[1], c->st[l + 1],
                           (const T*)c->e[l + 1], chalf);
                done = true;
            } else if (split) {
                launch_pdl(c, k_prolong_v<T, E, true>, vgrd, vblk, 0, L, st, e, m[0], m[1], c->st[l + 1],
                           (const T*)c->e[l + 1], A, rb.half, chalf);
                done = true;
            }
        }
        if (done) {
        } else if (vec)
            launch_pdl(c, k_prolong_v<T, E>, vgrd, vblk, 0, L, st, e, m[0], m[1], c->st[l + 1], (const T*)c->e[l + 1],
                       A, 0, 0);
        else if constexpr (kNative)
            launch_pdl(c, k_prolong<T>, full, blk, 0, L, st, e, m[0], m[1], c->st[l + 1], (const T*)c->e[l + 1]);
    }
    count(c);
    for (int s = 0; s < c->P.nu2; s++) sweep(0);
    return cudaGetLastError();
}

template <class T>
cudaError_t vcycle_level(es_ctx* c, int l, int warm) {
    if constexpr (std::is_same<T, float>::value)
        if (l == 0 && c->P.mg_storage == ES_MG_FP16) return vcycle_impl<float, __half>(c, l, warm);
    return vcycle_impl<T, T>(c, l, warm);
}

// (set before the V-cycle is captured into a graph).  The attribute belongs
// to the kernel, not to a context, so it is raised to the most any grid can
// need -- ty nxh <= 1024 and nxh <= 256 give at most kBulkSlots (2048 + 512)
// floats -- so that contexts of other sizes never lower it under each other.
void set_bulk_smem(es_ctx* c) {
    const size_t sm = bulk_smem_bytes(c);
    if (sm == 0 || c->bulk_smem_set) return;
    cudaFuncSetAttribute(k_smooth_rb_bulk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((size_t)kBulkSlots * (2048 + 512) * sizeof(float)));
    cudaGetLastError();
    // resident blocks per SM at this context's size (for the plane count)
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_smooth_rb_bulk<float>, 256, sm) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    c->bulk_blocks = b;
    c->bulk_smem_set = true;
}

// (the attribute belongs to the kernel: raised to the 200 KB every
// coarsest level that runs in one block fits, never lowered by a context
// with a smaller level)
template <class T>
void set_coarse_smem(const es_ctx* c) {
    size_t sm = coarse_smem_bytes(c, sizeof(T));
    if (sm > 48 * 1024 && sm <= 200 * 1024) {
        cudaFuncSetAttribute(k_coarse_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_coarse_lists<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
}

// The start of a solve when the float-float residual of the previous
// solve's potential is still in the finest right-hand side (colour-split,
// reduced forms) and every sphere has moved less than half a cell since
// then.  The residual changes only where a cell's stencil or boundary value
// changed: at the listed near-boundary cells (their boundary values and the
// spheres' surface charges), formed again by k_outer_residual_near_ff, and
// at the cells that flipped between obstacle and fluid (k_set, k_uncover)
// and their six neighbours (which covers the cells that stopped being
// near-boundary cells), formed here: 0 at obstacle cells.  A cell reached
// from several entries gets the same value each time.  gate: 1 when some
// sphere moved farther or the list overflowed (the full residual runs
// instead).
template <class M>
__global__ void __launch_bounds__(256) k_flip_patch(Grid g, ff diag0, WallFF wall, int pot_dir_mask,
                                                    const float* __restrict__ psi_hi,
                                                    const float* __restrict__ psi_lo,
                                                    const uint8_t* __restrict__ st0,
                                                    const int32_t* __restrict__ owner,
                                                    const float2* __restrict__ pbc,
                                                    const int* __restrict__ flips, const int* __restrict__ nflips,
                                                    int cap, float* __restrict__ r_out, M m,
                                                    const int* __restrict__ gate) {
    if (*gate != 0) return;
    const int n = *nflips < cap ? *nflips : cap;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 7 * n; i += gridDim.x * blockDim.x) {
        const int c = flips[i / 7], k = i % 7;
        int p3[3] = {c % nx, (c / nx) % ny, c / (nx * ny)};
        if (k > 0) {
            const int ax = (k - 1) >> 1, side = (k & 1) ? -1 : 1;
            const int n3 = ax == 0 ? nx : (ax == 1 ? ny : nz);
            int q = p3[ax] + side;
            if (q < 0 || q >= n3) {
                if (!g.per[ax]) continue;  // (beyond a wall: no cell)
                q = q < 0 ? q + n3 : q - n3;
            }
            p3[ax] = q;
        }
        const int cc = p3[0] + nx * (p3[1] + ny * p3[2]);
        const float v = (st0[cc] & ST_KIND) == ST_UNKNOWN
                            ? near_residual_ff(g, diag0, wall, pot_dir_mask, psi_hi, psi_lo, st0, owner, pbc, p3[0],
                                               p3[1], p3[2])
                            : 0.0f;
        r_out[m(cc, (p3[0] + p3[1] + p3[2]) & 1)] = v;
    }
}

// Sum of r^2 over the colour-split finest right-hand side, with the block
// layout and partial slots of k_outer_residual_ff<4, true> (zc planes a
// block), for the patched residual.  gate: 1 when the full residual runs
// instead.
__global__ void __launch_bounds__(256) k_rhs_norm_rb(Grid g, const float* __restrict__ r, int zc,
                                                     double* __restrict__ partial, const int* __restrict__ gate) {
    if (*gate != 0) return;
    __shared__ float swarp[8];
    const int half = (int)(g.N >> 1);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xs = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z0 = (int)blockIdx.z * zc;
    const int z1 = z0 + zc < nz ? z0 + zc : nz;
    float acc = 0.0f;
    if (xs < nx && y < ny)
        for (int z = z0; z < z1; z++) {
            const Q4<float> q = rb_ld4(r, half, xs + nx * (y + ny * z), (xs + y + z) & 1);
            acc = __fmaf_rn(q.v0, q.v0, acc);
            acc = __fmaf_rn(q.v1, q.v1, acc);
            acc = __fmaf_rn(q.v2, q.v2, acc);
            acc = __fmaf_rn(q.v3, q.v3, acc);
        }
    float v = acc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) swarp[threadIdx.y] = v;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; w++) tot += (double)swarp[w];
        partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = tot;
    }
}

// A local correction at a solve's start (after the patched residual).
// Between two solves the equation changes only around the few cells that
// flipped between obstacle and fluid, and there the start residual sits:
// the correction it asks for is a few screened point responses that decay
// like exp(-r kappa).  So the correction equation A e = r is first solved
// on the unknown cells within Chebyshev distance kLocalR of a flipped cell
// (e = 0 beyond them), by conjugate gradients in one block, before any
// V-cycle: psi += e there, r -= A e there and on the ring one cell further
// out, and the residual norm is updated by the change of r^2 over those
// cells.  The V-cycles then start from that residual (none when it is
// already below the tolerance).  Cells of the region carry bit 7 of their
// flag byte, ring cells bit 6, while the kernel runs.  Flipped cells closer
// than 2 kLocalR + 4 cells (Chebyshev, periodic images) form one cluster
// (k_local_clusters); one block corrects each cluster, and no two clusters'
// boxes share or touch a cell, so the blocks need no order; the norm takes
// their changes of r^2 in cluster order (k_local_norm).  gate: 1 when the
// full residual ran (a sphere moved far or the flip list overflowed); more
// than kLocalFlips flips leave the V-cycles alone, and a cluster whose
// region overflows its share of the scratch keeps its residual.
constexpr int kLocalR = 8;
constexpr int kLocalFlips = 16;
constexpr int kLocalIters = 40;
constexpr int kLocalCap = kLocalFlips * (2 * kLocalR + 3) * (2 * kLocalR + 3) * (2 * kLocalR + 3);
static_assert(kLocalCap == kLocalCells, "the scratch sized at creation");
constexpr int kLocalThreads = 1024;
constexpr int kLocalBox = (2 * kLocalR + 3) * (2 * kLocalR + 3) * (2 * kLocalR + 3);  // scratch cells a flip

// The clusters of the flipped cells, built by one thread: flips in cluster
// order, the cluster starts, the scratch base of each cluster (kLocalBox
// cells per flip), the cluster count, and room for each cluster's change of
// the squared norm.
struct LocalMeta {
    int n;
    int start[kLocalFlips + 1];
    int base[kLocalFlips];
    int flip[kLocalFlips];
    double delta[kLocalFlips];
};

static_assert(sizeof(LocalMeta) <= 1024, "the cluster table's allocation");

__global__ void k_local_clusters(Grid g, const int* __restrict__ flips, const int* __restrict__ nflips, int fcap,
                                 const int* __restrict__ gate, LocalMeta* meta) {
    if (threadIdx.x != 0) return;
    const int nf = *nflips;
    meta->n = 0;
    if (*gate != 0 || nf <= 0 || nf > kLocalFlips || nf > fcap) return;
    int cl[kLocalFlips];
    for (int i = 0; i < nf; i++) cl[i] = i;
    auto root = [&](int i) {
        while (cl[i] != i) i = cl[i];
        return i;
    };
    const int n3[3] = {g.nx, g.ny, g.nz};
    for (int i = 0; i < nf; i++)
        for (int j = i + 1; j < nf; j++) {
            const int a = flips[i], b = flips[j];
            const int pa[3] = {a % g.nx, (a / g.nx) % g.ny, a / (g.nx * g.ny)};
            const int pb[3] = {b % g.nx, (b / g.nx) % g.ny, b / (g.nx * g.ny)};
            int d = 0;
            for (int k = 0; k < 3; k++) {
                int dk = abs(pa[k] - pb[k]);
                if (g.per[k] && n3[k] - dk < dk) dk = n3[k] - dk;
                d = max(d, dk);
            }
            if (d <= 2 * kLocalR + 3) {
                const int ri = root(i), rj = root(j);
                if (ri != rj) cl[max(ri, rj)] = min(ri, rj);
            }
        }
    int n = 0, at = 0;
    for (int r = 0; r < nf; r++) {
        if (root(r) != r) continue;
        meta->start[n] = at;
        meta->base[n] = at * kLocalBox;
        for (int i = 0; i < nf; i++)
            if (root(i) == r) meta->flip[at++] = flips[i];
        meta->delta[n] = 0.0;
        n++;
    }
    meta->start[n] = at;
    meta->n = n;
}

// The residual norm after the local correction: the clusters' changes of
// r^2 in cluster order.
__global__ void k_local_norm(const LocalMeta* __restrict__ meta, double* norm) {
    if (threadIdx.x != 0 || meta->n == 0) return;
    double n2 = norm[0] * norm[0];
    for (int c = 0; c < meta->n; c++) n2 += meta->delta[c];
    norm[0] = sqrt(n2 > 0.0 ? n2 : 0.0);
}

__device__ __forceinline__ double block_sum_all(double v, double* sh) {
    v = block_sum(v, sh);
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = v;
    __syncthreads();
    v = sh[0];
    __syncthreads();
    return v;
}

// Visits the cells of the boxes of radius rb around the flipped cells
// (periodic axes wrapped, cells beyond a wall skipped); fn(cell, chebyshev
// distance).  Every thread of the block walks its share of each box.
template <class Fn>
__device__ __forceinline__ void local_boxes(const Level<float>& L, const int* flips, int nf, int rb, Fn&& fn) {
    const int nx = L.nx, ny = L.ny, nz = L.nz, side = 2 * rb + 1;
    const int vol = side * side * side;
    for (int f = 0; f < nf; f++) {
        const int c0 = flips[f];
        const int x0 = c0 % nx, y0 = (c0 / nx) % ny, z0 = c0 / (nx * ny);
        for (int t = threadIdx.x; t < vol; t += blockDim.x) {
            const int d3[3] = {t % side - rb, (t / side) % side - rb, t / (side * side) - rb};
            const int o3[3] = {x0, y0, z0}, n3[3] = {nx, ny, nz};
            int p3[3];
            bool ok = true;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                int v = o3[a] + d3[a];
                if (v < 0 || v >= n3[a]) {
                    if (!L.per[a]) {
                        ok = false;
                        break;
                    }
                    v = ((v % n3[a]) + n3[a]) % n3[a];
                }
                p3[a] = v;
            }
            if (!ok) continue;
            const int dist = max(abs(d3[0]), max(abs(d3[1]), abs(d3[2])));
            fn(p3[0] + nx * (p3[1] + ny * p3[2]), dist);
        }
    }
}

__global__ void __launch_bounds__(kLocalThreads) k_local_solve(Level<float> L, const uint8_t* __restrict__ st,
                                                               uint8_t* flags, LocalMeta* meta, float* r, float* e,
                                                               float* p, float* psi_hi, float* psi_lo, int* list_all,
                                                               float* rl_all, float* ec_all, float* q_all,
                                                               int half) {
    __shared__ int s_n[2];
    __shared__ int s_over;
    __shared__ double sh[32];
    const int cluster = blockIdx.x;
    if (cluster >= meta->n) return;  // (uniform over the block)
    const int f0 = meta->start[cluster], nf = meta->start[cluster + 1] - f0;
    const int* flips = meta->flip + f0;
    const int cap = nf * kLocalBox;  // this cluster's share of the scratch
    int* list = list_all + meta->base[cluster];
    float* rl = rl_all + meta->base[cluster];
    float* ec = ec_all + meta->base[cluster];
    float* q = q_all + meta->base[cluster];
    const RbMap rb{half};
    const int nx = L.nx, ny = L.ny;
    const float inv_h2 = 1.0f / L.h2;
    auto col = [&](int c) { return (c % nx + (c / nx) % ny + c / (nx * ny)) & 1; };
    auto word = [&](int c) { return reinterpret_cast<unsigned*>(flags + (c & ~3)); };
    if (threadIdx.x == 0) {
        s_n[0] = s_n[1] = 0;
        s_over = 0;
    }
    __syncthreads();
    // the region (distance <= kLocalR), then the ring (distance kLocalR + 1)
    // not in the region; each unknown cell listed once (its bit)
    for (int pass = 0; pass < 2; pass++) {
        const unsigned mark = pass == 0 ? 0x80u : 0x40u;
        local_boxes(L, flips, nf, kLocalR + pass, [&](int cc, int dist) {
            if (pass == 1 && dist != kLocalR + 1) return;
            if ((st[cc] & ST_KIND) != ST_UNKNOWN) return;
            const int sh8 = 8 * (cc & 3);
            const unsigned old = atomicOr(word(cc), mark << sh8);
            if ((old >> sh8) & (pass == 0 ? 0x80u : 0xC0u)) return;  // (listed already, or in the region)
            const int i = atomicAdd(&s_n[1], 1);
            if (i < cap)
                list[i] = cc;
            else
                s_over = 1;
        });
        __syncthreads();
        if (pass == 0 && threadIdx.x == 0) s_n[0] = s_n[1];
        __syncthreads();
    }
    const int ni = min(s_n[0], cap), nt = min(s_n[1], cap);
    if (!s_over) {
        // e = p = 0 on the listed cells (the ring keeps 0: A restricted to the region)
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            const int cc = list[i], cl = col(cc);
            e[rb(cc, cl)] = 0.0f;
            p[rb(cc, cl)] = 0.0f;
        }
        __syncthreads();
        double rr = 0.0, old_sq = 0.0;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            const int cc = list[i];
            const float v = r[rb(cc, col(cc))];
            old_sq += (double)v * v;
            if (i < ni) {
                rl[i] = v;
                ec[i] = 0.0f;
                p[rb(cc, col(cc))] = v;
                rr += (double)v * v;
            }
        }
        rr = block_sum_all(rr, sh);
        old_sq = block_sum_all(old_sq, sh);
        const double rr0 = rr;
        for (int it = 0; it < kLocalIters && rr > 1e-6 * rr0 && rr > 0.0; it++) {
            double pq = 0.0;
            for (int i = threadIdx.x; i < ni; i += blockDim.x) {
                const int cc = list[i];
                const int x = cc % nx, y = (cc / nx) % ny, z = cc / (nx * ny);
                float dg, off;
                level_stencil<float, true, float, RbMap>(L, st, p, x, y, z, st[cc], dg, off,
                                                         EAcc<float, float>{1.0f, 1.0f}, rb);
                const float pv = p[rb(cc, col(cc))];
                const float qv = (dg * pv - off) * inv_h2;
                q[i] = qv;
                pq += (double)pv * qv;
            }
            pq = block_sum_all(pq, sh);
            if (!(pq > 0.0)) break;
            const double alpha = rr / pq;
            double rn = 0.0;
            for (int i = threadIdx.x; i < ni; i += blockDim.x) {
                const int cc = list[i];
                ec[i] += (float)alpha * p[rb(cc, col(cc))];
                rl[i] -= (float)alpha * q[i];
                rn += (double)rl[i] * rl[i];
            }
            rn = block_sum_all(rn, sh);  // (also: every thread is done reading p)
            const float beta = (float)(rn / rr);
            for (int i = threadIdx.x; i < ni; i += blockDim.x) {
                const int cc = list[i];
                float* pp = p + rb(cc, col(cc));
                *pp = rl[i] + beta * *pp;
            }
            __syncthreads();
            rr = rn;
        }
        // psi += e on the region; e in place for the residual
        for (int i = threadIdx.x; i < ni; i += blockDim.x) {
            const int cc = list[i];
            e[rb(cc, col(cc))] = ec[i];
            const ff v = ff_add_f({psi_hi[cc], psi_lo[cc]}, ec[i]);
            psi_hi[cc] = v.hi;
            psi_lo[cc] = v.lo;
        }
        __syncthreads();
        // r -= A e on the region and the ring (e = 0 beyond the region: a
        // neighbour counts only if it carries the region's bit)
        double new_sq = 0.0;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            const int cc = list[i];
            const int x = cc % nx, y = (cc / nx) % ny, z = cc / (nx * ny);
            float dg, off0;
            level_stencil<float, false, float, RbMap>(L, st, e, x, y, z, st[cc], dg, off0,
                                                      EAcc<float, float>{1.0f, 1.0f}, rb);
            const int c3[3] = {x, y, z}, n3[3] = {L.nx, L.ny, L.nz}, stride[3] = {1, nx, nx * ny};
            const int ncol = 1 - ((x + y + z) & 1);
            float off = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int sd = -1; sd <= 1; sd += 2) {
                    int v = c3[a] + sd;
                    if (v < 0 || v >= n3[a]) {
                        if (!L.per[a]) continue;
                        v = v < 0 ? v + n3[a] : v - n3[a];
                    }
                    const int nb = cc + (v - c3[a]) * stride[a];
                    if ((st[nb] & ST_KIND) != ST_UNKNOWN) continue;
                    if ((flags[nb] & 0x80u) == 0) continue;  // (e = 0 there)
                    off += e[rb(nb, ncol)];
                }
            const float ev = i < ni ? ec[i] : 0.0f;
            float* rp = r + rb(cc, col(cc));
            const float rv = *rp - (dg * ev - off) * inv_h2;
            *rp = rv;
            new_sq += (double)rv * rv;
        }
        new_sq = block_sum_all(new_sq, sh);
        if (threadIdx.x == 0) meta->delta[cluster] = new_sq - old_sq;
    }
    __syncthreads();
    // clear the bits (every box cell: also those an overflow left unlisted)
    local_boxes(L, flips, nf, kLocalR + 1, [&](int cc, int) { atomicAnd(word(cc), ~(0xC0u << (8 * (cc & 3)))); });
}

}  // namespace

// Grid of a marching residual pass over a level of nz planes with (gx, gy)
// blocks per plane: zc planes per block, about eight blocks per SM in all
// (up to 16 planes each), and no more blocks than partial-sum slots.
static void res_march_grid(const es_ctx* c, int gx, int gy, int nz, int& gz, int& zc) {
    const long long plane = (long long)gx * gy;
    zc = (int)(plane * nz / (8LL * c->n_sm));
    zc = zc < 1 ? 1 : (zc > 16 ? 16 : zc);
    const long long slots = (long long)res_partial_slots(c->g.nx, c->g.ny, c->red_blocks);
    const long long planes = slots / plane;  // >= 1
    if ((nz + zc - 1) / zc > planes) zc = (int)((nz + planes - 1) / planes);
    gz = (nz + zc - 1) / zc;
}

// Algorithmic bytes per cell: psi (8: double, or float-float) and the state
// byte in, r out (8 as double, 4 as the float right-hand side).
cudaError_t launch_outer_residual(es_ctx* c, bool patch) {
    const double diag0 = 6.0 + c->S.kappa * c->S.kappa;
    patch = patch && mixed(c) && c->rb0;
    // (bytes: the full residual's; a patched start moves r once, 4 a cell, plus the listed cells)
    ProfScope ps(c, patch ? "residual_patch" : "outer_residual", -1,
                 (double)c->g.N * (patch ? 4.0 : (mixed(c) ? 13.0 : 17.0)));
    if (mixed(c)) {
        WallFF wall;
        int mask = 0;
        for (int f = 0; f < 6; f++) {
            const ff v = ff_from_double(2.0 * c->S.pot_val[f]);
            wall.hi[f] = v.hi;
            wall.lo[f] = v.lo;
            if (c->S.pot_bc[f] == ES_POT_DIRICHLET) mask |= 1 << f;
        }
        const int W = (c->g.nx % 4) == 0 ? 4 : 1;
        const int gx = (c->g.nx / W + 31) / 32, gy = (c->g.ny + 7) / 8;
        int gz, zc;
        res_march_grid(c, gx, gy, c->g.nz, gz, zc);
        const dim3 grd(gx, gy, gz), blk(32, 8);
        const dim3 ngrd(near_grid_x(c), 2 * kNearSegs);
        const ff d0 = ff_from_double(diag0);
        float* r = (float*)c->rhs[0];
        // patch: the full residual only if the mapping flagged a sphere that
        // moved half a cell or more (the gate), else the patched one
        const int* gate = patch ? c->d_moved : nullptr;
        if (c->rb0) {
            // r goes to the colour-split right-hand side of the finest level
            const RbMap rb{(int)(c->g.N / 2)};
            k_outer_residual_near_ff<RbMap><<<ngrd, 256, 0, c->stream>>>(
                c->g, d0, wall, mask, c->psi32, c->psi_lo, c->st[0], c->owner, (const float2*)c->pbc,
                c->near_list[0], c->near_count, c->near_cap[0], r, rb);
            k_outer_residual_ff<4, true><<<grd, blk, 0, c->stream>>>(c->g, d0, c->psi32, c->psi_lo, c->st[0], r,
                                                                      c->partial, zc, gate);
            if (patch) {
                k_flip_patch<RbMap><<<2 * c->n_sm, 256, 0, c->stream>>>(
                    c->g, d0, wall, mask, c->psi32, c->psi_lo, c->st[0], c->owner, (const float2*)c->pbc,
                    c->flip_list, c->flip_count, c->flip_cap, r, rb, c->d_moved);
                k_rhs_norm_rb<<<grd, blk, 0, c->stream>>>(c->g, r, zc, c->partial, c->d_moved);
                count(c, 2);
            }
        } else {
            k_outer_residual_near_ff<NatMap><<<ngrd, 256, 0, c->stream>>>(
                c->g, d0, wall, mask, c->psi32, c->psi_lo, c->st[0], c->owner, (const float2*)c->pbc,
                c->near_list[0], c->near_count, c->near_cap[0], r, NatMap{});
            if (W == 4)
                k_outer_residual_ff<4, false><<<grd, blk, 0, c->stream>>>(c->g, d0, c->psi32, c->psi_lo, c->st[0],
                                                                           r, c->partial, zc, nullptr);
            else
                k_outer_residual_ff<1, false><<<grd, blk, 0, c->stream>>>(c->g, d0, c->psi32, c->psi_lo, c->st[0],
                                                                           r, c->partial, zc, nullptr);
        }
        k_finalize_norm<<<1, 1024, 0, c->stream>>>(c->partial, gx * gy * gz, c->d_norm);
        count(c, 3);
        if (patch && c->local_list) {
            // the local correction around the flipped cells (k_local_solve), one block a cluster
            LocalMeta* meta = (LocalMeta*)c->local_meta;
            k_local_clusters<<<1, 32, 0, c->stream>>>(c->g, c->flip_list, c->flip_count, c->flip_cap, c->d_moved,
                                                      meta);
            k_local_solve<<<kLocalFlips, kLocalThreads, 0, c->stream>>>(
                level_desc<float>(c, 0), c->st[0], c->flags, meta, r, (float*)c->e[0], (float*)c->e2[0],
                c->psi32, c->psi_lo, c->local_list, c->local_f, c->local_f + kLocalCap, c->local_f + 2 * kLocalCap,
                (int)(c->g.N / 2));
            k_local_norm<<<1, 32, 0, c->stream>>>(meta, c->d_norm);
            count(c, 3);
        }
        // (the mapping raises the flag again when a sphere moves far, and
        // lists the cells that flip from here on)
        cudaError_t err = cudaMemsetAsync(c->d_moved, 0, sizeof(int), c->stream);
        if (err == cudaSuccess) err = cudaMemsetAsync(c->flip_count, 0, sizeof(int), c->stream);
        if (err != cudaSuccess) return err;
        return cudaGetLastError();
    }
    const double k2 = c->S.kappa * c->S.kappa;
    if (c->P.phi_t > 0.0)
        k_outer_residual<true><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            c->g, c->S, diag0, k2, c->P.phi_t, c->dk, c->psi, c->st[0], c->owner, c->part, c->kind,
            (double*)c->rhs[0], c->partial);
    else
        k_outer_residual<false><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            c->g, c->S, diag0, k2, 0.0, nullptr, c->psi, c->st[0], c->owner, c->part, c->kind,
            (double*)c->rhs[0], c->partial);
    k_finalize_norm<<<1, 1024, 0, c->stream>>>(c->partial, c->red_blocks, c->d_norm);
    count(c, 2);
    return cudaGetLastError();
}

namespace {
cudaError_t vcycle_direct(es_ctx* c, int warm) {
    if (mixed(c)) return vcycle_level<float>(c, 0, warm);
    return vcycle_level<double>(c, 0, warm);
}
}  // namespace

// The V-cycle's launches depend only on the context's shapes, buffers and
// on `warm` (device-side data such as the near-cell lists and their counts
// are read at run time), so each of the two sequences is captured once into
// a CUDA graph and replayed: the many small coarse-level kernels then follow
// each other without a host launch apiece.  Launched directly instead while
// per-kernel profiling brackets launches with events, with the fused sweep
// (it swaps iterate buffers between cycles), with the FP16 correction (its
// scale changes per correction), on the legacy default stream (no capture
// there), or after a capture failed.
cudaError_t launch_vcycle(es_ctx* c, int warm) {
    if (mixed(c))
        set_coarse_smem<float>(c);
    else
        set_coarse_smem<double>(c);
    set_bulk_smem(c);
    const bool graph = !c->prof && !c->vgraph_off && c->stream != nullptr &&
                       c->P.smoother == ES_SMOOTH_TWO_PASS && c->P.mg_storage == ES_MG_NATIVE;
    if (!graph) return vcycle_direct(c, warm);
    const int w = warm ? 1 : 0;
    if (!c->vgraph[w]) {
        const unsigned long long before = c->launches;
        cudaError_t err = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) {
            cudaGetLastError();
            c->vgraph_off = true;
            return vcycle_direct(c, warm);
        }
        const cudaError_t cerr = vcycle_direct(c, warm);
        cudaGraph_t gph = nullptr;
        err = cudaStreamEndCapture(c->stream, &gph);
        cudaGraphExec_t ge = nullptr;
        if (cerr == cudaSuccess && err == cudaSuccess && gph)
            err = cudaGraphInstantiate(&ge, gph, 0);
        if (gph) cudaGraphDestroy(gph);
        // (the launches counted while capturing are the graph's kernels; they
        // run at each replay)
        const unsigned long long captured = c->launches - before;
        c->launches = before;
        if (cerr != cudaSuccess || err != cudaSuccess || !ge) {
            cudaGetLastError();
            c->vgraph_off = true;
            return vcycle_direct(c, warm);
        }
        c->vgraph[w] = ge;
        c->vgraph_kernels[w] = captured;
    }
    count(c, c->vgraph_kernels[w]);
    return cudaGraphLaunch(c->vgraph[w], c->stream);
}

// Algorithmic bytes per cell: e (s) and the state byte in, psi (8) in and out.
cudaError_t launch_correct(es_ctx* c) {
    const int N = (int)c->g.N;
    const double es = c->P.mg_storage == ES_MG_FP16 ? 2.0 : (mixed(c) ? 4.0 : 8.0);
    ProfScope ps(c, "correct", -1, (double)N * (es + 1.0 + 16.0));
    if (mixed(c)) {
        const int n4 = (N >> 2) > 0 ? (N >> 2) : 1;
        if (c->P.mg_storage == ES_MG_FP16)
            k_correct_ff<__half><<<(n4 + 255) / 256, 256, 0, c->stream>>>(
                N, c->st[0], (const __half*)c->e[0], c->psi32, c->psi_lo,
                EAcc<float, __half>{c->e_scale, 1.0f / c->e_scale});
        else if (c->rb0)
            k_correct_ff<float, true><<<(n4 + 255) / 256, 256, 0, c->stream>>>(
                N, c->st[0], (const float*)c->e[0], c->psi32, c->psi_lo, EAcc<float, float>{1.0f, 1.0f}, c->g.nx,
                c->g.ny);
        else
            k_correct_ff<float><<<(n4 + 255) / 256, 256, 0, c->stream>>>(
                N, c->st[0], (const float*)c->e[0], c->psi32, c->psi_lo, EAcc<float, float>{1.0f, 1.0f});
    } else {
        k_correct<<<(N + 255) / 256, 256, 0, c->stream>>>(N, c->st[0], (const double*)c->e[0], c->psi);
    }
    count(c);
    return cudaGetLastError();
}

// The FP32 residual update of the colour-split finest level (reduced
// forms); correct: with the correction psi += e in the same pass (else
// k_correct_ff applies it).  Algorithmic bytes per cell: e (4), r in and out
// (8), the state byte, and with the correction psi in and out (16).
cudaError_t launch_residual_update(es_ctx* c, bool correct) {
    Level<float> L = level_desc<float>(c, 0);
    const int N = (int)c->g.N, nxh = L.nx / 2;
    ProfScope ps(c, correct ? "residual_update_correct" : "residual_update", -1, (double)N * (correct ? 29.0 : 13.0));
    float* scratch = (float*)c->e2[0];
    const dim3 ngrd(near_grid_x(c), 2 * kNearSegs);
    k_near_residual<float, float, RbMap><<<ngrd, 256, 0, c->stream>>>(
        L, c->st[0], (const float*)c->rhs[0], (const float*)c->e[0], c->near_list[0], c->near_count,
        c->near_cap[0], 1.0f / L.h2, scratch, EAcc<float, float>{1.0f, 1.0f}, RbMap{N / 2});
    const int gx = (nxh / 4 + 31) / 32, gy = (L.ny + 7) / 8;
    int gz, zc;
    res_march_grid(c, gx, gy, L.nz, gz, zc);
    if (correct)
        k_residual_update_rb<true><<<dim3(gx, gy, gz), dim3(32, 8), 0, c->stream>>>(
            L, 1.0f / L.h2, c->st[0], (float*)c->rhs[0], (const float*)c->e[0], scratch, N / 2, c->partial, zc,
            c->psi32, c->psi_lo);
    else
        k_residual_update_rb<false><<<dim3(gx, gy, gz), dim3(32, 8), 0, c->stream>>>(
            L, 1.0f / L.h2, c->st[0], (float*)c->rhs[0], (const float*)c->e[0], scratch, N / 2, c->partial, zc,
            nullptr, nullptr);
    k_finalize_norm<<<1, 1024, 0, c->stream>>>(c->partial, gx * gy * gz, c->d_norm);
    count(c, 3);
    return cudaGetLastError();
}

cudaError_t launch_split_psi(es_ctx* c, const double* src) {
    const int N = (int)c->g.N;
    k_split_psi<<<(N + 255) / 256, 256, 0, c->stream>>>(N, src, c->psi32, c->psi_lo);
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_join_psi(es_ctx* c, double* dst) {
    const int N = (int)c->g.N;
    k_join_psi<<<(N + 255) / 256, 256, 0, c->stream>>>(N, c->psi32, c->psi_lo, dst);
    count(c);
    return cudaGetLastError();
}

// The reduced forms on grids with nx % 4 == 0 evaluate f_b inside the
// stream-collide (body_force_iso at interior fluid cells, the stored field
// at cells next to obstacles and walls): the solve only marks the body force
// as derived from psi.
bool fb_fused(const es_ctx* c) { return mixed(c) && c->g.nx % 4 == 0; }

// f_b of the fluid cells with a non-fluid D3Q19 neighbour (the D3Q7
// ghost-value gradient; list of cells), into the stored field.
cudaError_t launch_body_force_near(es_ctx* c) {
    const Grid& g = c->g;
    const double* E = c->P.E_ext;
    const double k2e = c->S.kappa * c->S.kappa * c->S.eps;
    WallF wall2;
    for (int f = 0; f < 6; f++) wall2.v2[f] = (float)(2.0 * c->S.pot_val[f]);
    ProfScope ps(c, "body_force_near", -1, 0.0);
    k_body_force_near<<<dim3(near_grid_x(c), kNearSegs), 256, 0, c->stream>>>(
        g, c->S, (float)E[0], (float)E[1], (float)E[2], (float)k2e, c->psi32, c->owner, c->st[0],
        (const float2*)c->pbc, wall2, c->bf_list, c->bf_count, c->bf_cap, (float*)c->fb);
    count(c);
    return cudaGetLastError();
}

// Algorithmic bytes per cell: psi as the kernel reads it (float in MIXED32,
// double in FP64) and the flag byte in, f_b (3 s) out.  Writes the whole
// field (the fused forms call it when the field is read).
cudaError_t launch_body_force_full(es_ctx* c) {
    const Grid& g = c->g;
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny, g.nz);
    const double s = mixed(c) ? 4.0 : 8.0;
    const double* E = c->P.E_ext;
    const double k2e = c->S.kappa * c->S.kappa * c->S.eps;
    WallF wall2;
    for (int f = 0; f < 6; f++) wall2.v2[f] = (float)(2.0 * c->S.pot_val[f]);
    if (fb_fused(c)) {
        {
            ProfScope ps(c, "body_force", -1, (double)g.N * (s + 1.0 + 3.0 * s));
            dim3 vgrd((g.nx / 4 + 31) / 32, (g.ny + 7) / 8, g.nz);
            k_body_force_v<<<vgrd, dim3(32, 8), 0, c->stream>>>(g, (float)E[0], (float)E[1], (float)E[2],
                                                                (float)k2e, c->psi32, c->flags, (float*)c->fb);
            count(c);
        }
        return launch_body_force_near(c);
    }
    ProfScope ps(c, "body_force", -1, (double)g.N * (s + 1.0 + 3.0 * s));
    if (mixed(c))
        k_body_force<float, float><<<grd, blk, 0, c->stream>>>(g, c->S, (float)E[0], (float)E[1], (float)E[2],
                                                               (float)k2e, 0.0f, c->psi32, c->flags, c->owner, c->part,
                                                               c->kind, c->st[0], (const float2*)c->pbc, wall2,
                                                               (float*)c->fb);
    else
        k_body_force<double, double><<<grd, blk, 0, c->stream>>>(g, c->S, E[0], E[1], E[2], k2e, c->P.phi_t,
                                                                 c->psi, c->flags,
                                                                 c->owner, c->part, c->kind, c->st[0], nullptr,
                                                                 wall2, (double*)c->fb);
    count(c);
    return cudaGetLastError();
}

// The body force after a solve: computed and stored here (FP64, and reduced
// forms with nx % 4 != 0), or left to the stream-collide (fb_fused).
cudaError_t launch_body_force(es_ctx* c) {
    if (fb_fused(c)) {
        c->fb_lazy = true;
        return cudaSuccess;
    }
    c->fb_lazy = false;
    return launch_body_force_full(c);
}

// Before the stored field is read (FB, U and the stream-collide's cells next
// to obstacles): the values of a body force that is evaluated on the fly.
cudaError_t materialize_body_force(es_ctx* c) { return c->fb_lazy ? launch_body_force_full(c) : cudaSuccess; }

}  // namespace es
