// es_lbm.cu -- fused stream-collide (a7), momentum-exchange force/torque (a8)
// and rigid-body update (a9); Sec. 4.1, Sec. 4.2, Sec. 5.7.
//
// Stream-collide is a single pull sweep over a structure-of-arrays PDF
// field: a thread per cell gathers f_q(x) = f~_q(x - e_q) from the 19
// streams (a warp reads 32 consecutive cells of each stream; the +-x
// shifted streams are one element off and are served by the same L1/L2
// sectors), collides in registers and writes its 19 populations.  Cells
// next to an obstacle or a wall (F_NEAR19) take the moving bounce-back of
// Eq. LBMMovWall instead of the pull for the affected directions.
//
// MIXED32 stores f_q - w_q in float: the collision is linear in f, and the
// weights cancel in every term except the density, which becomes 1 + sum.
#include <type_traits>

#include "es_device.cuh"

namespace es {

namespace {

// Base pointers of the 19 source and destination streams, so that an access
// is a 32-bit cell offset from a base (no 64-bit products in the kernel).
template <class S>
struct Streams {
    const S* src[19];
    S* dst[19];
};

// Float copy of the particle state used by the FP32 stream-collide (centre,
// velocity, angular velocity), so that its moving-wall term needs no FP64.
__global__ void k_particles_f32(int np, const DParticle* __restrict__ part, float* __restrict__ pf) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    for (int a = 0; a < 3; a++) {
        pf[12 * p + a] = (float)part[p].x[a];
        pf[12 * p + 3 + a] = (float)part[p].v[a];
        pf[12 * p + 6 + a] = (float)part[p].w[a];
    }
}

// A population whose pull source lies beyond a non-periodic face (walls
// half-way outside the first and last layer): the direction and cell it is
// taken from.  No-slip face: resting bounce-back, the cell's own population
// of the opposite direction.  Free-slip (every crossed face free-slip):
// specular reflection; the population arriving with e_q left the fluid cell
// s = x - (the components of e_q parallel to the crossed faces) in the
// direction with the crossed components reversed.  An obstacle cell at s
// falls back to bounce-back.  Either direction has the weight of q.
struct WallSrc {
    int q;
    long long cell;
};

__device__ __forceinline__ WallSrc wall_source(const Grid& g, int slip_faces, const int32_t* __restrict__ owner,
                                               int x, int y, int z, int q, long long c) {
    const int cv[3] = {cx(q), cy(q), cz(q)};
    const int p[3] = {x, y, z};
    const int n[3] = {g.nx, g.ny, g.nz};
    int m[3], s[3];
    bool slip = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int v = p[a] - cv[a];
        if (cv[a] != 0 && !g.per[a] && (v < 0 || v >= n[a])) {
            slip = slip && ((slip_faces >> (2 * a + (v >= n[a] ? 1 : 0))) & 1);
            m[a] = -cv[a];
            s[a] = p[a];
        } else {
            m[a] = cv[a];
            s[a] = v < 0 ? v + n[a] : (v >= n[a] ? v - n[a] : v);
        }
    }
    if (slip) {
        const long long sc = lin(g, s[0], s[1], s[2]);
        if (owner[sc] < 0) {
            int qm = 0;
#pragma unroll
            for (int k = 1; k < 19; k++)
                if (cx(k) == m[0] && cy(k) == m[1] && cz(k) == m[2]) qm = k;
            return WallSrc{qm, sc};
        }
    }
    return WallSrc{opp(q), c};
}

// TRT collision of one cell from its pulled populations f (working values)
// and its body force plus acceleration: the moments (Eq. MacroscopVel) with
// the modified velocity (Eq. modified_velocity), the even and odd parts of
// Eq. TRTOp with the incompressible equilibrium (Eq. EqPDF_TRT) and Luo's
// forcing (Eq. LBE_forcetermLuo); put(q, v) receives each post-collision
// value.  Every stream-collide kernel calls this one function, so all give
// the same bits.
template <class C, class Put>
__device__ __forceinline__ void collide(const C (&f)[19], C fx, C fy, C fz, C lam_e, C lam_o, Put&& put) {
    // moments (Eq. MacroscopVel) with the modified velocity (Eq. modified_velocity)
    C rho = (C)0, jx = (C)0, jy = (C)0, jz = (C)0;
#pragma unroll
    for (int q = 0; q < 19; q++) {
        rho += f[q];
        if (cx(q)) jx += cx(q) > 0 ? f[q] : -f[q];
        if (cy(q)) jy += cy(q) > 0 ? f[q] : -f[q];
        if (cz(q)) jz += cz(q) > 0 ? f[q] : -f[q];
    }
    // in the shifted form rho holds rho - 1; w_q * rho below is then the
    // shifted equilibrium directly
    const C ux = jx + (C)0.5 * fx, uy = jy + (C)0.5 * fy, uz = jz + (C)0.5 * fz;
    const C uu = ux * ux + uy * uy + uz * uz;
    const C uf = ux * fx + uy * fy + uz * fz;
    const C ae = (C)1 + (C)0.5 * lam_e, ao = (C)1 + (C)0.5 * lam_o;

    // rest population: even part only
    {
        const C w0 = (C)wq(0);
        const C eq0 = w0 * (rho - (C)1.5 * uu);
        const C F0 = w0 * ((C)-3 * uf);
        put(0, f[0] + lam_e * (f[0] - eq0) + ae * F0);
    }
    // pairs (q, q+9): TRT split into even and odd parts (Eq. TRTOp, Eq. EqPDF_TRT)
#pragma unroll
    for (int q = 1; q <= 9; q++) {
        const C w = (C)wq(q);
        const C cu = (C)cx(q) * ux + (C)cy(q) * uy + (C)cz(q) * uz;
        const C cf = (C)cx(q) * fx + (C)cy(q) * fy + (C)cz(q) * fz;
        const C eq_e = w * (rho + (C)4.5 * cu * cu - (C)1.5 * uu);
        const C eq_o = w * (C)3 * cu;
        const C fe = (C)0.5 * (f[q] + f[q + 9]);
        const C fo = (C)0.5 * (f[q] - f[q + 9]);
        // Luo's term (Eq. LBE_forcetermLuo) split: even w(9 cu cf - 3 u.f), odd 3 w cf,
        // with the (1 + lambda/2) factors that go with the modified velocity
        const C Fe = w * ((C)9 * cu * cf - (C)3 * uf);
        const C Fo = w * (C)3 * cf;
        const C even = lam_e * (fe - eq_e) + ae * Fe;
        const C odd = lam_o * (fo - eq_o) + ao * Fo;
        put(q, f[q] + even + odd);
        put(q + 9, f[q + 9] + even - odd);
    }
}

// The electric body force evaluated inside the stream-collide (reduced
// forms): psi (the float potential), E_ext and kappa^2 eps.
struct FbPsi {
    const float* psi;
    float Ex, Ey, Ez, k2e;
};

// SLIP: the grid has free-slip faces (a separate instance, so that the
// common no-slip/periodic form keeps its register count).  FBPSI: the body
// force of an interior fluid cell (no obstacle or wall among its D3Q19
// neighbours) is formed here from the potential at the cell and its 18
// neighbours (body_force_iso, Sec. 5.6), so f_b makes no round trip through
// HBM: the cell reads 4 bytes of psi (the neighbours' come from cache)
// instead of 12 of stored f_b.  Cells next to obstacles or walls read the
// stored field (their D3Q7 ghost-value gradient, k_body_force_near).
template <class S, bool SLIP, bool FBPSI, bool EARLY, class C = typename Store<S>::C>
__device__ __forceinline__ void lbm_cell(const Grid& g, const Streams<S>& P, const uint8_t* __restrict__ flags,
                                         const int32_t* __restrict__ owner, const DParticle* __restrict__ part,
                                         const float* __restrict__ partf, const C* __restrict__ fb, C ax, C ay,
                                         C az, C lam_e, C lam_o, int slip_faces, const FbPsi& fp, int x, int y,
                                         int z) {
    using St = Store<S>;
    const unsigned N = (unsigned)g.N;
    const int nx = g.nx, nxy = g.nx * g.ny;
    const int c = x + nx * (y + g.ny * z);
    const uint8_t fl = flags[c];
    // The pull sources x - e_q with every axis wrapped: in bounds for every
    // cell, and the true sources of all cells but the few next to an
    // obstacle or a wall.  EARLY: they are loaded before the cell's flags
    // arrive, so the two loads do not follow one another (obstacle cells
    // load and drop them, and cells next to an obstacle keep those of their
    // fluid neighbours, the same cells, and replace the others below);
    // otherwise each path loads what it needs after the flags (fewer live
    // registers, for the persistent batched kernel).  Same values either way.
    const int sx[3] = {(x == nx - 1 ? 0 : x + 1) - x, 0, (x == 0 ? nx - 1 : x - 1) - x};
    const int sy[3] = {((y == g.ny - 1 ? 0 : y + 1) - y) * nx, 0, ((y == 0 ? g.ny - 1 : y - 1) - y) * nx};
    const int sz[3] = {((z == g.nz - 1 ? 0 : z + 1) - z) * nxy, 0, ((z == 0 ? g.nz - 1 : z - 1) - z) * nxy};
    C f[19];
    auto pull = [&]() {
#pragma unroll
        for (int q = 0; q < 19; q++) {
            const int s_ = c + sx[1 + cx(q)] + sy[1 + cy(q)] + sz[1 + cz(q)];
            f[q] = St::ld(q, __ldg(P.src[q] + s_));
        }
    };
    if constexpr (EARLY) pull();
    if (fl & F_SOLID) return;  // obstacle cells are not updated

    C fx, fy, fz;  // body force (Sec. 5.6) plus the uniform acceleration
    if (!(fl & F_NEAR19)) {
        // all 18 pull sources are fluid cells inside the (periodic) domain
        if constexpr (FBPSI) {
            // psi(x + d) at offset sx[1 - dx] + sy[1 - dy] + sz[1 - dz]
            const float* ps = fp.psi + c;
            const Psi19 p{__ldg(ps),
                          __ldg(ps + sx[0]),
                          __ldg(ps + sx[2]),
                          __ldg(ps + sy[0]),
                          __ldg(ps + sy[2]),
                          __ldg(ps + sz[0]),
                          __ldg(ps + sz[2]),
                          __ldg(ps + sx[0] + sy[0]),
                          __ldg(ps + sx[2] + sy[2]),
                          __ldg(ps + sx[0] + sy[2]),
                          __ldg(ps + sx[2] + sy[0]),
                          __ldg(ps + sx[0] + sz[0]),
                          __ldg(ps + sx[2] + sz[2]),
                          __ldg(ps + sx[0] + sz[2]),
                          __ldg(ps + sx[2] + sz[0]),
                          __ldg(ps + sy[0] + sz[0]),
                          __ldg(ps + sy[2] + sz[2]),
                          __ldg(ps + sy[0] + sz[2]),
                          __ldg(ps + sy[2] + sz[0])};
            float f0, f1, f2;
            body_force_iso(p, fp.Ex, fp.Ey, fp.Ez, fp.k2e, f0, f1, f2);
            fx = f0 + ax;
            fy = f1 + ay;
            fz = f2 + az;
        } else {
            fx = fb[c] + ax;
            fy = fb[N + c] + ay;
            fz = fb[2u * N + c] + az;
        }
        if constexpr (!EARLY) pull();
    } else {
        fx = fb[c] + ax;
        fy = fb[N + c] + ay;
        fz = fb[2u * N + c] + az;
        if constexpr (!EARLY) f[0] = St::ld(0, P.src[0][c]);
#pragma unroll
        for (int q = 1; q < 19; q++) {
            long long nb;
            if (!neighbour(g, x, y, z, -cx(q), -cy(q), -cz(q), nb)) {
                if constexpr (SLIP) {
                    const WallSrc w = wall_source(g, slip_faces, owner, x, y, z, q, c);
                    f[q] = St::ld(q, P.src[w.q][w.cell]);
                } else {
                    f[q] = St::ld(opp(q), P.src[opp(q)][c]);  // resting no-slip wall: bounce back
                }
                continue;
            }
            const int o = owner[nb];
            if (o < 0) {  // a fluid source: the value pulled above
                if constexpr (!EARLY) f[q] = St::ld(q, P.src[q][nb]);
                continue;
            }
            // moving bounce-back (Eq. LBMMovWall): the population sent from x
            // towards the surface cell returns with 2 w_q rho_0 (c_q . u_s)/c_s^2
            if constexpr (sizeof(C) == 4) {
                // FP32 form: lever arm from the float copy of the particle
                const float* pf = partf + 12 * o;
                float r[3] = {(float)x + 0.5f - (float)cx(q) - pf[0], (float)y + 0.5f - (float)cy(q) - pf[1],
                              (float)z + 0.5f - (float)cz(q) - pf[2]};
                const float Lw[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
#pragma unroll
                for (int a = 0; a < 3; a++)
                    if (g.per[a]) {
                        if (r[a] > 0.5f * Lw[a]) r[a] -= Lw[a];
                        if (r[a] < -0.5f * Lw[a]) r[a] += Lw[a];
                    }
                const float u0 = pf[3] + (pf[7] * r[2] - pf[8] * r[1]);
                const float u1 = pf[4] + (pf[8] * r[0] - pf[6] * r[2]);
                const float u2 = pf[5] + (pf[6] * r[1] - pf[7] * r[0]);
                const float cu = (float)cx(q) * u0 + (float)cy(q) * u1 + (float)cz(q) * u2;
                f[q] = St::ld(opp(q), P.src[opp(q)][c]) + (float)(6.0 * wq(q)) * cu;
            } else {
                int bx = x - cx(q), by = y - cy(q), bz = z - cz(q);
                bx = bx < 0 ? bx + g.nx : (bx >= g.nx ? bx - g.nx : bx);
                by = by < 0 ? by + g.ny : (by >= g.ny ? by - g.ny : by);
                bz = bz < 0 ? bz + g.nz : (bz >= g.nz ? bz - g.nz : bz);
                double us[3];
                surface_velocity(g, part[o].x, part[o].v, part[o].w, bx, by, bz, us);
                const double cu = cx(q) * us[0] + cy(q) * us[1] + cz(q) * us[2];
                f[q] = St::ld(opp(q), P.src[opp(q)][c]) + (C)(6.0 * wq(q) * cu);
            }
        }
    }

    collide<C>(f, fx, fy, fz, lam_e, lam_o, [&](int q, C v) { P.dst[q][c] = St::st(q, v); });
}

// One thread per cell; a block covers blockDim.x cells of blockDim.y rows
// (the shape is a parameter: es_params.lbm_block).
// (the reduced forms cap a thread at 48 registers, 1,280 threads per SM: with
// the pull loads issued ahead of the flag test, 40 registers spill and 64
// leave too few threads; both measured slower)
template <class S, bool SLIP, bool FBPSI = false, class C = typename Store<S>::C>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 3 : 5) k_lbm(Grid g, const Streams<S> P, const uint8_t* __restrict__ flags,
                                             const int32_t* __restrict__ owner, const DParticle* __restrict__ part,
                                             const float* __restrict__ partf, const C* __restrict__ fb, C ax, C ay,
                                             C az, C lam_e, C lam_o, int slip_faces, FbPsi fp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    lbm_cell<S, SLIP, FBPSI, true>(g, P, flags, owner, part, partf, fb, ax, ay, az, lam_e, lam_o, slip_faces, fp, x, y,
                             z);
}

// Several resident runs stepped by one persistent launch (es_lbm_step_batch):
// a work table of the runs' fields and parameters, passed by value, and a
// flat index of tiles of 32 cells x 4 rows over all runs (run r owns tiles
// tile0[r] .. tile0[r+1]-1).  Blocks of 128 threads stride over the tiles;
// each cell runs the same lbm_cell as k_lbm, so a run gives the same bits
// alone and in a batch.
constexpr int kBatchTileX = 32, kBatchTileY = 4;

template <class S>
struct BatchRun {
    using C = typename Store<S>::C;
    Grid g;
    Streams<S> P;
    const uint8_t* flags;
    const int32_t* owner;
    const DParticle* part;
    const float* partf;
    const C* fb;
    C ax, ay, az, lam_e, lam_o;
    FbPsi fp;
    int lazy;        // f_b from psi inside the stream-collide
    int tiles_x;     // tiles per row of tiles: ceil(nx / 32)
    int tiles_y;     // rows of tiles per plane: ceil(ny / 4)
    long long tile0; // first tile of the run
};

template <class S>
struct BatchTable {
    BatchRun<S> r[ES_LBM_BATCH_MAX];
    int n;
    long long ntiles;
};

template <class S>
__global__ void __launch_bounds__(kBatchTileX * kBatchTileY, sizeof(S) == 8 ? 6 : 8)
    k_lbm_batch(const __grid_constant__ BatchTable<S> T) {
    const int tx = threadIdx.x % kBatchTileX, ty = threadIdx.x / kBatchTileX;
    int r = 0;
    for (long long t = blockIdx.x; t < T.ntiles; t += gridDim.x) {
        while (r + 1 < T.n && T.r[r + 1].tile0 <= t) r++;
        const BatchRun<S>& R = T.r[r];
        const long long loc = t - R.tile0;
        const int bx = (int)(loc % R.tiles_x);
        const long long rest = loc / R.tiles_x;
        const int by = (int)(rest % R.tiles_y), z = (int)(rest / R.tiles_y);
        const int x = bx * kBatchTileX + tx, y = by * kBatchTileY + ty;
        if (x >= R.g.nx || y >= R.g.ny) continue;
        if constexpr (std::is_same<typename Store<S>::C, float>::value) {
            if (R.lazy) {
                lbm_cell<S, false, true, false>(R.g, R.P, R.flags, R.owner, R.part, R.partf, R.fb, R.ax, R.ay, R.az,
                                         R.lam_e, R.lam_o, 0, R.fp, x, y, z);
                continue;
            }
        }
        lbm_cell<S, false, false, false>(R.g, R.P, R.flags, R.owner, R.part, R.partf, R.fb, R.ax, R.ay, R.az, R.lam_e,
                                  R.lam_o, 0, R.fp, x, y, z);
    }
}

// Momentum exchange (Eq. LBMhydrodynForce): one block per sphere.  Each
// link x_F -> x_F + e_q into the sphere adds [2 f~_q(x_F) - 2 w_q (c_q . u_s)/c_s^2] c_q
// and the torque (x_s - X) x dF.  The box around the sphere is scanned 256
// cells at a time; the links found are compacted into shared memory in
// (thread, direction) order by a block prefix sum and then summed one link
// per thread, so the FP64 arithmetic (1/64 rate on GB300) runs on dense
// warps instead of on divergent lanes.  Fixed order: deterministic.
constexpr int kForceThreads = 256;

template <class S>
__global__ void __launch_bounds__(kForceThreads) k_forces(Grid g, const DParticle* __restrict__ part,
                                                          const int32_t* __restrict__ owner,
                                                          const uint8_t* __restrict__ flags,
                                                          const S* __restrict__ src, double Ex, double Ey, double Ez,
                                                          const double* __restrict__ mapped, double* F, double* T) {
    __shared__ int s_cell[kForceThreads * 18];
    __shared__ uint8_t s_q[kForceThreads * 18];
    __shared__ int s_warp[kForceThreads / 32];
    __shared__ double sh[32];
    const int p = blockIdx.x;
    const DParticle P = part[p];
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) axis_range(g, a, P.x[a], P.x[a], P.R, 1, lo[a], hi[a]);
    const int sx = hi[0] - lo[0] + 1, sy = hi[1] - lo[1] + 1, sz = hi[2] - lo[2] + 1;
    // A link runs from a fluid cell to a cell of p within sqrt 2, and p's
    // cells are those within R of its centre at the last mapping, so only
    // cells between R - 1 and R + 1.5 of that centre are scanned (FP32
    // distances; the bounds are far outside their rounding).
    BallF ball;
    ball.init(g, mapped + 9 * p, P.R, lo, hi);
    const float rin = (float)P.R - 1.0f, rout = (float)P.R + 1.5f;
    const float in2 = rin > 0.0f ? rin * rin : -1.0f, out2 = rout * rout;
    const int n = sx * sy * sz;
    const size_t ps = (size_t)g.ps;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int base = 0; base < n; base += kForceThreads) {
        const int t = base + threadIdx.x;
        unsigned mask = 0;
        int c = 0;
        bool scan = t < n;
        if (scan && ball.ok) {
            const float d2 = ball.d2(t % sx, (t / sx) % sy, t / (sx * sy));
            scan = d2 >= in2 && d2 <= out2;
        }
        if (scan) {
            const int tx = t % sx, tyz = t / sx;
            const int x = wrap_coord(lo[0] + tx, g.nx);
            const int y = wrap_coord(lo[1] + tyz % sy, g.ny);
            const int z = wrap_coord(lo[2] + tyz / sy, g.nz);
            c = x + g.nx * (y + g.ny * z);
            if (flags[c] & F_NEAR19) {
#pragma unroll
                for (int q = 1; q < 19; q++) {
                    long long nb;
                    if (neighbour(g, x, y, z, cx(q), cy(q), cz(q), nb) && owner[nb] == p) mask |= 1u << q;
                }
            }
        }
        // block-wide exclusive prefix sum of the link counts
        const int cnt = __popc(mask);
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        int woff = 0, total = 0;
        for (int w = 0; w < kForceThreads / 32; w++) {
            if (w < wid) woff += s_warp[w];
            total += s_warp[w];
        }
        int off = woff + incl - cnt;
        while (mask) {
            const int q = __ffs(mask) - 1;
            mask &= mask - 1;
            s_cell[off] = c;
            s_q[off] = (uint8_t)q;
            off++;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < total; i += kForceThreads) {
            const int cc = s_cell[i], q = s_q[i];
            const int x = cc % g.nx, yz = cc / g.nx;
            const int y = yz % g.ny, z = yz / g.ny;
            int qx = 0, qy = 0, qz = 0;
#pragma unroll
            for (int k = 1; k < 19; k++)
                if (k == q) {
                    qx = cx(k);
                    qy = cy(k);
                    qz = cz(k);
                }
            const int bx = wrap_coord(x + qx, g.nx), by = wrap_coord(y + qy, g.ny), bz = wrap_coord(z + qz, g.nz);
            const double r0 = cell_disp(g, 0, bx, P.x[0]);
            const double r1 = cell_disp(g, 1, by, P.x[1]);
            const double r2 = cell_disp(g, 2, bz, P.x[2]);
            const double us0 = P.v[0] + (P.w[1] * r2 - P.w[2] * r1);
            const double us1 = P.v[1] + (P.w[2] * r0 - P.w[0] * r2);
            const double us2 = P.v[2] + (P.w[0] * r1 - P.w[1] * r0);
            const double cu = qx * us0 + qy * us1 + qz * us2;
            const double w = (q <= 3 || (q >= 10 && q <= 12)) ? 1.0 / 18.0 : 1.0 / 36.0;
            const double fq = Store<S>::to_f(q, src[q * ps + cc]);
            const double m = 2.0 * fq - 6.0 * w * cu;
            const double d0 = m * qx, d1 = m * qy, d2 = m * qz;
            acc[0] += d0;
            acc[1] += d1;
            acc[2] += d2;
            acc[3] += r1 * d2 - r2 * d1;
            acc[4] += r2 * d0 - r0 * d2;
            acc[5] += r0 * d1 - r1 * d0;
        }
        __syncthreads();
    }
    const double E[3] = {Ex, Ey, Ez};
    for (int k = 0; k < 6; k++) {
        double s = block_sum(acc[k], sh);
        if (threadIdx.x == 0) {
            if (k < 3)
                F[3 * p + k] = s + P.qeff * E[k];  // F_C = q E_ext (Sec. 5.6)
            else
                T[3 * p + k - 3] = s;
        }
    }
}

// Momentum exchange of the reduced forms (float or FP16 populations, stored
// as deviations f - w_q).  Same links and sums as k_forces, arranged so that
// no FP64 arithmetic runs per link (GB300's FP64 rate is a small fraction
// of its FP32 rate).  With f~ = w_q + dev the link term is
// [2 w_q + m'] c_q, m' = 2 dev - 6 w_q (c_q . u_s):
//  * the m' part (small) is summed in FP32 per thread, with lever arms in
//    FP32, and over the block in float-float;
//  * the 2 w_q part is summed exactly: per direction, the number of links
//    and the integer sums of the surface cells' coordinates (relative to the
//    box origin, unwrapped), from which thread 0 forms sum 2 w_q c_q and
//    sum 2 w_q (x_s - X) x c_q in FP64 at the end.
// Near-surface scan as in k_forces (cells between R - 1 and R + 1.5 of the
// centre at the last mapping).  Deterministic: fixed summation order.
template <class S>
__global__ void __launch_bounds__(kForceThreads) k_forces_f32(Grid g, const DParticle* __restrict__ part,
                                                              const int32_t* __restrict__ owner,
                                                              const uint8_t* __restrict__ flags,
                                                              const S* __restrict__ src, double Ex, double Ey,
                                                              double Ez, const double* __restrict__ mapped,
                                                              double* F, double* T) {
    using St = Store<S>;
    constexpr int kTile = 4096;  // (with the link lists below, within 48 KB of static shared memory)
    __shared__ int tile[kTile];
    __shared__ int s_cell[kForceThreads * 18];
    __shared__ uint8_t s_q[kForceThreads * 18];
    __shared__ int s_warp[kForceThreads / 32];
    __shared__ int s_lo[3], s_n[3];
    __shared__ BallF s_ball;
    __shared__ float s_X[3], s_V[3], s_W[3], s_band[2];
    __shared__ int s_cnt[19], s_sum[19][3];
    __shared__ float s_red[kForceThreads / 32][12];
    const int p = blockIdx.x;
    if (threadIdx.x == 0) {
        const DParticle& P = part[p];
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            axis_range(g, a, P.x[a], P.x[a], P.R, 1, lo[a], hi[a]);
            s_lo[a] = lo[a];
            s_n[a] = hi[a] - lo[a] + 1;
            // centre relative to the box origin's cell centre: r = i - s_X for
            // the cell with local index i (exact to FP32 rounding of s_X)
            s_X[a] = (float)(P.x[a] - ((double)lo[a] + 0.5));
            s_V[a] = (float)P.v[a];
            s_W[a] = (float)P.w[a];
        }
        s_ball.init(g, mapped + 9 * p, P.R, lo, hi);
        const float rin = (float)P.R - 1.0f, rout = (float)P.R + 1.5f;
        s_band[0] = rin > 0.0f ? rin * rin : -1.0f;
        s_band[1] = rout * rout;
    }
    if (threadIdx.x < 19) {
        s_cnt[threadIdx.x] = 0;
        s_sum[threadIdx.x][0] = s_sum[threadIdx.x][1] = s_sum[threadIdx.x][2] = 0;
    }
    __syncthreads();
    const int sx = s_n[0], sy = s_n[1], sz = s_n[2];
    const int n = sx * sy * sz;
    const BallF ball = s_ball;
    const OwnerTile TL{{sx, sy, sz}};
    const bool use_tile = TL.fits(kTile);
    if (use_tile) {
        const int lo3[3] = {s_lo[0], s_lo[1], s_lo[2]};
        load_owner_tile(g, owner, lo3, TL, tile);
        __syncthreads();
    }
    const float in2 = s_band[0], out2 = s_band[1];
    const float Xr[3] = {s_X[0], s_X[1], s_X[2]}, V[3] = {s_V[0], s_V[1], s_V[2]}, W[3] = {s_W[0], s_W[1], s_W[2]};
    const int L[3] = {g.nx, g.ny, g.nz};
    const size_t ps = (size_t)g.ps;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    BoxWalk bw;
    bw.start(threadIdx.x, kForceThreads, sx, sy);
    for (int base = 0; base < n; base += kForceThreads, bw.next()) {
        const int t = base + threadIdx.x;
        unsigned mask = 0;
        int c = 0;
        bool scan = t < n;
        if (scan && ball.ok) {
            const float d2 = ball.d2(bw.i, bw.j, bw.k);
            scan = d2 >= in2 && d2 <= out2;
        }
        if (scan) {
            if (use_tile) {
                const int ti = TL.at(bw.i, bw.j, bw.k);
                if (tile[ti] < 0 && tile[ti] != kOwnerOutside) {
#pragma unroll
                    for (int q = 1; q < 19; q++)
                        if (tile[ti + TL.step(q)] == p) mask |= 1u << q;
                }
            } else {
                const int x = wrap1(s_lo[0] + bw.i, g.nx);
                const int y = wrap1(s_lo[1] + bw.j, g.ny);
                const int z = wrap1(s_lo[2] + bw.k, g.nz);
                const int cg = x + g.nx * (y + g.ny * z);
                if (flags[cg] & F_NEAR19) {
#pragma unroll
                    for (int q = 1; q < 19; q++) {
                        long long nb;
                        if (neighbour(g, x, y, z, cx(q), cy(q), cz(q), nb) && owner[nb] == p) mask |= 1u << q;
                    }
                }
            }
            c = bw.i | (bw.j << 10) | (bw.k << 20);  // local indices of x_F (a box is < 1024 cells a side)
        }
        const int cnt = __popc(mask);
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        int woff = 0, total = 0;
        for (int w = 0; w < kForceThreads / 32; w++) {
            if (w < wid) woff += s_warp[w];
            total += s_warp[w];
        }
        int off = woff + incl - cnt;
        while (mask) {
            const int q = __ffs(mask) - 1;
            mask &= mask - 1;
            s_cell[off] = c;
            s_q[off] = (uint8_t)q;
            off++;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < total; i += kForceThreads) {
            const int pk = s_cell[i], q = s_q[i];
            const int li[3] = {pk & 1023, (pk >> 10) & 1023, pk >> 20};
            const int cc = wrap1(s_lo[0] + li[0], g.nx) +
                           g.nx * (wrap1(s_lo[1] + li[1], g.ny) + g.ny * wrap1(s_lo[2] + li[2], g.nz));
            int qv[3] = {0, 0, 0};
#pragma unroll
            for (int k = 1; k < 19; k++)
                if (k == q) {
                    qv[0] = cx(k);
                    qv[1] = cy(k);
                    qv[2] = cz(k);
                }
            // surface cell x_s = x_F + c_q in the box's unwrapped frame
            // (minimum image where a periodic box spans the whole axis)
            int rel[3];
            float r[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                int u = li[a] + qv[a];
                if (g.per[a]) {
                    if ((float)u - Xr[a] > 0.5f * (float)L[a]) u -= L[a];
                    if ((float)u - Xr[a] < -0.5f * (float)L[a]) u += L[a];
                }
                rel[a] = u;
                r[a] = (float)u - Xr[a];
            }
            const float us0 = V[0] + (W[1] * r[2] - W[2] * r[1]);
            const float us1 = V[1] + (W[2] * r[0] - W[0] * r[2]);
            const float us2 = V[2] + (W[0] * r[1] - W[1] * r[0]);
            const float cu = (float)qv[0] * us0 + (float)qv[1] * us1 + (float)qv[2] * us2;
            const float w = (q <= 3 || (q >= 10 && q <= 12)) ? 1.0f / 18.0f : 1.0f / 36.0f;
            float dev;  // f~ - w_q
            if constexpr (std::is_same<S, __half>::value)
                dev = __half2float(src[q * ps + cc]) * (w * (float)(1.0 / kHalfScale));  // (Store<__half>::ld in FP32)
            else
                dev = St::ld(q, src[q * ps + cc]);
            const float m = 2.0f * dev - 6.0f * w * cu;
            const float d0 = m * (float)qv[0], d1 = m * (float)qv[1], d2 = m * (float)qv[2];
            acc[0] += d0;
            acc[1] += d1;
            acc[2] += d2;
            acc[3] += r[1] * d2 - r[2] * d1;
            acc[4] += r[2] * d0 - r[0] * d2;
            acc[5] += r[0] * d1 - r[1] * d0;
            atomicAdd(&s_cnt[q], 1);
            atomicAdd(&s_sum[q][0], rel[0]);
            atomicAdd(&s_sum[q][1], rel[1]);
            atomicAdd(&s_sum[q][2], rel[2]);
        }
        __syncthreads();
    }
    // block sum of the six FP32 partials in float-float (fixed order)
    ff v[6];
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = {acc[k], 0.0f};
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const ff u = {__shfl_down_sync(0xffffffffu, v[k].hi, o), __shfl_down_sync(0xffffffffu, v[k].lo, o)};
            v[k] = ff_add(v[k], u);
        }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; k++) {
            s_red[wid][2 * k] = v[k].hi;
            s_red[wid][2 * k + 1] = v[k].lo;
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        const DParticle& P = part[p];
        double sum[6];
        for (int k = 0; k < 6; k++) {
            ff a = {s_red[0][2 * k], s_red[0][2 * k + 1]};
            for (int w = 1; w < kForceThreads / 32; w++) a = ff_add(a, ff{s_red[w][2 * k], s_red[w][2 * k + 1]});
            sum[k] = (double)a.hi + (double)a.lo;
        }
        // the 2 w_q part: sum 2 w_q c_q and sum 2 w_q (x_s - X) x c_q, with
        // x_s - X = rel + (lo + 1/2 - X)
        double off[3];
        for (int a = 0; a < 3; a++) off[a] = (double)s_lo[a] + 0.5 - P.x[a];
        for (int q = 1; q < 19; q++) {
            if (s_cnt[q] == 0) continue;
            const double w2 = 2.0 * ((q <= 3 || (q >= 10 && q <= 12)) ? 1.0 / 18.0 : 1.0 / 36.0);
            const double nq = (double)s_cnt[q];
            const double c3[3] = {(double)cx(q), (double)cy(q), (double)cz(q)};
            double rs[3];  // sum over the links of x_s - X
            for (int a = 0; a < 3; a++) rs[a] = (double)s_sum[q][a] + nq * off[a];
            sum[0] += w2 * nq * c3[0];
            sum[1] += w2 * nq * c3[1];
            sum[2] += w2 * nq * c3[2];
            sum[3] += w2 * (rs[1] * c3[2] - rs[2] * c3[1]);
            sum[4] += w2 * (rs[2] * c3[0] - rs[0] * c3[2]);
            sum[5] += w2 * (rs[0] * c3[1] - rs[1] * c3[0]);
        }
        const double E[3] = {Ex, Ey, Ez};
        for (int k = 0; k < 3; k++) {
            F[3 * p + k] = sum[k] + P.qeff * E[k];  // F_C = q E_ext (Sec. 5.6)
            T[3 * p + k] = sum[3 + k];
        }
    }
}

// Semi-implicit Euler, dt = 1 (the integrator is a reading: the paper
// leaves it to the pe engine).
__global__ void k_advance(int np, DParticle* part, const double* F, const double* T, int px, int py, int pz,
                          double Lx, double Ly, double Lz) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    DParticle& P = part[p];
    const int per[3] = {px, py, pz};
    const double L[3] = {Lx, Ly, Lz};
    for (int a = 0; a < 3; a++) {
        P.v[a] += F[3 * p + a] / P.mass;
        P.x[a] += P.v[a];
        P.w[a] += T[3 * p + a] / P.inertia;
        if (per[a]) {
            if (P.x[a] >= L[a]) P.x[a] -= L[a];
            if (P.x[a] < 0.0) P.x[a] += L[a];
        }
    }
}

template <class S>
__global__ void k_fill_rest(int N, size_t ps, S* a, S* b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i >= N) return;
    const S v = Store<S>::rest(q);
    a[q * ps + i] = v;
    b[q * ps + i] = v;
}

// PDFs are exchanged densely (19 x N doubles) and stored with stride ps.
template <class S>
__global__ void k_get_pdf(long long N, long long ps, const S* src, double* dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 19 * N) return;
    int q = (int)(i / N);
    dst[i] = Store<S>::to_f(q, src[(long long)q * ps + (i - (long long)q * N)]);
}

template <class S>
__global__ void k_set_pdf(long long N, long long ps, const double* src, S* dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 19 * N) return;
    int q = (int)(i / N);
    dst[(long long)q * ps + (i - (long long)q * N)] = Store<S>::from_f(q, src[i]);
}

template <class S, class C = typename Store<S>::C>
__global__ void k_moments(long long N, long long ps, const S* f, const C* fb, double ax, double ay, double az,
                          double* rho, double* u) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    double r = 0.0, j0 = 0.0, j1 = 0.0, j2 = 0.0;
    for (int q = 0; q < 19; q++) {
        double v = Store<S>::to_f(q, f[(long long)q * ps + c]);
        r += v;
        j0 += cx(q) * v;
        j1 += cy(q) * v;
        j2 += cz(q) * v;
    }
    // collision keeps rho and adds exactly f_b, so u = sum c f - f_b / 2
    if (rho) rho[c] = r;
    if (u) {
        u[c] = j0 - 0.5 * ((double)fb[c] + ax);
        u[N + c] = j1 - 0.5 * ((double)fb[N + c] + ay);
        u[2 * N + c] = j2 - 0.5 * ((double)fb[2 * N + c] + az);
    }
}

template <class S>
__global__ void k_copy_fb(long long n, const S* a, double* b) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

template <class S>
__global__ void k_load_fb(long long n, const double* a, S* b) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (S)a[i];
}

template <class S, class C = typename Store<S>::C>
__global__ void k_gather(int which, long long N, long long ps, const long long* idx, int n, const S* cur, const S* last,
                         const C* fb, const double* psi, const float* psi_hi, const float* psi_lo,
                         const int32_t* owner, const uint8_t* flags, double ax, double ay, double az, double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long c = idx[i];
    switch (which) {
    case ES_FIELD_PSI: out[i] = psi ? psi[c] : (double)psi_hi[c] + (double)psi_lo[c]; break;
    case ES_FIELD_OWNER: out[i] = (double)owner[c]; break;
    case ES_FIELD_FLAGS: out[i] = (double)flags[c]; break;
    case ES_FIELD_FB:
        for (int k = 0; k < 3; k++) out[(long long)k * n + i] = (double)fb[k * N + c];
        break;
    case ES_FIELD_PDF:
    case ES_FIELD_PDF_LAST: {
        const S* f = which == ES_FIELD_PDF ? cur : last;
        for (int q = 0; q < 19; q++) out[(long long)q * n + i] = Store<S>::to_f(q, f[q * ps + c]);
        break;
    }
    case ES_FIELD_RHO:
    case ES_FIELD_U: {
        double r = 0.0, j0 = 0.0, j1 = 0.0, j2 = 0.0;
        for (int q = 0; q < 19; q++) {
            double v = Store<S>::to_f(q, cur[q * ps + c]);
            r += v;
            j0 += cx(q) * v;
            j1 += cy(q) * v;
            j2 += cz(q) * v;
        }
        if (which == ES_FIELD_RHO) {
            out[i] = r;
        } else {
            out[i] = j0 - 0.5 * ((double)fb[c] + ax);
            out[(long long)n + i] = j1 - 0.5 * ((double)fb[N + c] + ay);
            out[2LL * n + i] = j2 - 0.5 * ((double)fb[2 * N + c] + az);
        }
        break;
    }
    }
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <class S>
Streams<S> streams(const es_ctx* c) {
    Streams<S> P;
    const S* src = (const S*)c->pdf[c->cur];
    S* dst = (S*)c->pdf[1 - c->cur];
    for (int q = 0; q < 19; q++) {
        P.src[q] = src + (size_t)q * (size_t)c->g.ps;
        P.dst[q] = dst + (size_t)q * (size_t)c->g.ps;
    }
    return P;
}

// Calls fn with a value of the context's PDF storage type (double, float or
// __half) so that a generic lambda can instantiate the kernel for it.
template <class Fn>
void dispatch_store(const es_ctx* c, Fn&& fn) {
    if (c->P.precision == ES_MIXED16)
        fn(__half{});
    else if (mixed(c))
        fn(0.0f);
    else
        fn(0.0);
}

// The stream-collide's block shape (es_params.lbm_block; 0 = 32 x 4: a warp
// per row segment and four rows a block, so that the rows y +- 1 of psi the
// fused body force reads are mostly in the block's own L1; measured at 512^3
// 3.95 ms against 4.14 ms for 128 x 1).
dim3 lbm_block(const es_ctx* c) {
    if (c->P.lbm_block[0] <= 0) return dim3(32, 4);
    return dim3(c->P.lbm_block[0], c->P.lbm_block[1] > 0 ? c->P.lbm_block[1] : 1);
}

cudaError_t launch_lbm(es_ctx* c) {
    const Grid& g = c->g;
    const dim3 blk = lbm_block(c);
    const dim3 grd((g.nx + blk.x - 1) / blk.x, (g.ny + blk.y - 1) / blk.y, g.nz);
    const double* a = c->P.accel;
    if (mixed(c) && c->np > 0) {
        k_particles_f32<<<(c->np + 127) / 128, 128, 0, c->stream>>>(c->np, c->part, c->partf);
        count(c);
    }
    // the body force evaluated in the stream-collide: first the stored values
    // of the cells next to obstacles and walls
    const bool lazy = c->fb_lazy;
    if (lazy) {
        const cudaError_t e = launch_body_force_near(c);
        if (e != cudaSuccess) return e;
    }
    const double k2e = c->S.kappa * c->S.kappa * c->S.eps;
    const FbPsi fp{c->psi32, (float)c->P.E_ext[0], (float)c->P.E_ext[1], (float)c->P.E_ext[2], (float)k2e};
    dispatch_store(c, [&](auto tag) {
        using S = decltype(tag);
        using C = typename Store<S>::C;
        // algorithmic bytes per cell: 19 populations in and out, f_b (3 C)
        // or psi (4) and the flag byte in
        ProfScope ps(c, "lbm", -1, (double)g.N * (38.0 * sizeof(S) + (lazy ? 4.0 : 3.0 * sizeof(C)) + 1.0));
        auto run = [&](auto slip, auto fused) {
            k_lbm<S, decltype(slip)::value, decltype(fused)::value><<<grd, blk, 0, c->stream>>>(
                g, streams<S>(c), c->flags, c->owner, c->part, c->partf, (const C*)c->fb, (C)a[0], (C)a[1], (C)a[2],
                (C)c->lambda_e, (C)c->lambda_o, c->slip, fp);
        };
        using T_ = std::true_type;
        using F_ = std::false_type;
        if constexpr (std::is_same<C, float>::value) {
            if (lazy) {
                if (c->slip)
                    run(T_{}, T_{});
                else
                    run(F_{}, T_{});
                return;
            }
        }
        if (c->slip)
            run(T_{}, F_{});
        else
            run(F_{}, F_{});
    });
    count(c);
    return cudaGetLastError();
}

// The stream-collide of n contexts (same precision and device, no
// free-slip faces; checked by the caller) in one launch on cs[0]'s stream,
// ordered after each context's pending work and before its later work by
// events.  Each context's per-run preparation (the float particle copy, the
// body force at cells next to obstacles) runs on its own stream first.
cudaError_t launch_lbm_batch(es_ctx* const* cs, int n) {
    cudaStream_t bs = cs[0]->stream;
    for (int i = 0; i < n; i++) {
        es_ctx* c = cs[i];
        if (mixed(c) && c->np > 0) {
            k_particles_f32<<<(c->np + 127) / 128, 128, 0, c->stream>>>(c->np, c->part, c->partf);
            count(c);
        }
        if (c->fb_lazy) {
            const cudaError_t e = launch_body_force_near(c);
            if (e != cudaSuccess) return e;
        }
        if (!c->ev_sync) {
            const cudaError_t e = cudaEventCreateWithFlags(&c->ev_sync, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        if (i > 0) {
            cudaError_t e = cudaEventRecord(c->ev_sync, c->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, c->ev_sync, 0);
            if (e != cudaSuccess) return e;
        }
    }
    cudaError_t err = cudaSuccess;
    dispatch_store(cs[0], [&](auto tag) {
        using S = decltype(tag);
        using C = typename Store<S>::C;
        BatchTable<S> T;
        long long tiles = 0;
        double cells = 0.0;
        for (int i = 0; i < n; i++) {
            es_ctx* c = cs[i];
            BatchRun<S>& R = T.r[i];
            R.g = c->g;
            R.P = streams<S>(c);
            R.flags = c->flags;
            R.owner = c->owner;
            R.part = c->part;
            R.partf = c->partf;
            R.fb = (const C*)c->fb;
            R.ax = (C)c->P.accel[0];
            R.ay = (C)c->P.accel[1];
            R.az = (C)c->P.accel[2];
            R.lam_e = (C)c->lambda_e;
            R.lam_o = (C)c->lambda_o;
            const double k2e = c->S.kappa * c->S.kappa * c->S.eps;
            R.fp = FbPsi{c->psi32, (float)c->P.E_ext[0], (float)c->P.E_ext[1], (float)c->P.E_ext[2], (float)k2e};
            R.lazy = c->fb_lazy ? 1 : 0;
            R.tiles_x = (c->g.nx + kBatchTileX - 1) / kBatchTileX;
            R.tiles_y = (c->g.ny + kBatchTileY - 1) / kBatchTileY;
            R.tile0 = tiles;
            tiles += (long long)R.tiles_x * R.tiles_y * c->g.nz;
            cells += (double)c->g.N;
        }
        T.n = n;
        T.ntiles = tiles;
        const long long cap = (long long)cs[0]->n_sm * 16;
        const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
        ProfScope ps(cs[0], "lbm_batch", -1, cells * (38.0 * sizeof(S) + 4.0 + 1.0));
        k_lbm_batch<S><<<grid, kBatchTileX * kBatchTileY, 0, bs>>>(T);
        count(cs[0]);
        err = cudaGetLastError();
    });
    if (err != cudaSuccess) return err;
    err = cudaEventRecord(cs[0]->ev_sync, bs);
    for (int i = 1; i < n && err == cudaSuccess; i++) err = cudaStreamWaitEvent(cs[i]->stream, cs[0]->ev_sync, 0);
    return err;
}

cudaError_t launch_forces(es_ctx* c) {
    if (c->np == 0) return cudaSuccess;
    const double* E = c->P.E_ext;
    int src = c->last_src >= 0 ? c->last_src : c->cur;
    ProfScope ps(c, "forces", -1, 0.0);
    dispatch_store(c, [&](auto tag) {
        using S = decltype(tag);
        // (the FP32 form packs box-local indices in 10 bits per axis)
        double rmax = 0.0;
        for (double r : c->h_R) rmax = r > rmax ? r : rmax;
        const bool small_boxes = 2.0 * rmax + 8.0 < 1024.0;
        if (std::is_same<S, double>::value || !small_boxes)
            k_forces<S><<<c->np, kForceThreads, 0, c->stream>>>(c->g, c->part, c->owner, c->flags,
                                                                (const S*)c->pdf[src], E[0], E[1], E[2], c->mapped,
                                                                c->F, c->T);
        else
            k_forces_f32<S><<<c->np, kForceThreads, 0, c->stream>>>(c->g, c->part, c->owner, c->flags,
                                                                    (const S*)c->pdf[src], E[0], E[1], E[2],
                                                                    c->mapped, c->F, c->T);
    });
    count(c);
    return cudaGetLastError();
}

// A new particle state from the host: position, velocities, zeta, q and the
// charge of the Coulomb force (Eq. SurfChrgZetaRelationDebHuck for a zeta
// sphere) replace the record's; the surface charge density found by the last
// mapping stays until the next one recomputes it, and the mass and moment of
// inertia follow from the fixed radius.  In the MIXED32 form the sphere's
// boundary value (2 zeta, or sigma / eps) is split into float-float as the
// mapping does.
__global__ void k_set_particles(const double* __restrict__ in, DParticle* part, const int* kind, double eps,
                                float* pbc, int np) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double* s = in + 12 * p;
    DParticle& d = part[p];
    for (int a = 0; a < 3; a++) {
        d.x[a] = s[a];
        d.v[a] = s[3 + a];
        d.w[a] = s[6 + a];
    }
    d.zeta = s[9];
    d.q = s[10];
    d.qeff = s[11];
    if (pbc) {
        const ff v = ff_from_double(kind[p] == ES_KIND_ZETA ? 2.0 * d.zeta : d.sigma / eps);
        pbc[2 * p] = v.hi;
        pbc[2 * p + 1] = v.lo;
    }
}

cudaError_t launch_set_particles(es_ctx* c) {
    if (c->np == 0) return cudaSuccess;
    k_set_particles<<<blocks_for(c->np, 128), 128, 0, c->stream>>>(c->pstage, c->part, c->kind, c->S.eps, c->pbc,
                                                                   c->np);
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_advance(es_ctx* c) {
    if (c->np == 0) return cudaSuccess;
    ProfScope ps(c, "advance", -1, 0.0);
    k_advance<<<blocks_for(c->np, 128), 128, 0, c->stream>>>(c->np, c->part, c->F, c->T, c->g.per[0], c->g.per[1],
                                                             c->g.per[2], (double)c->g.nx, (double)c->g.ny,
                                                             (double)c->g.nz);
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_fill_rest(es_ctx* c) {
    const int N = (int)c->g.N;
    dim3 grd((N + 255) / 256, 19);
    dispatch_store(c, [&](auto tag) {
        using S = decltype(tag);
        k_fill_rest<S><<<grd, 256, 0, c->stream>>>(N, (size_t)c->g.ps, (S*)c->pdf[0], (S*)c->pdf[1]);
    });
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_get_pdf(es_ctx* c, int buf, double* dst) {
    long long n = 19 * c->g.N;
    dispatch_store(c, [&](auto tag) {
        using S = decltype(tag);
        k_get_pdf<S><<<blocks_for(n, 256), 256, 0, c->stream>>>(c->g.N, c->g.ps, (const S*)c->pdf[buf], dst);
    });
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_set_pdf(es_ctx* c, const double* src) {
    long long n = 19 * c->g.N;
    dispatch_store(c, [&](auto tag) {
        using S = decltype(tag);
        k_set_pdf<S><<<blocks_for(n, 256), 256, 0, c->stream>>>(c->g.N, c->g.ps, src, (S*)c->pdf[c->cur]);
    });
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_get_moments(es_ctx* c, double* rho, double* u) {
    const cudaError_t err = materialize_body_force(c);
    if (err != cudaSuccess) return err;
    const double* a = c->P.accel;
    dispatch_store(c, [&](auto tag) {
        using S = decltype(tag);
        using C = typename Store<S>::C;
        k_moments<S><<<blocks_for(c->g.N, 256), 256, 0, c->stream>>>(c->g.N, c->g.ps, (const S*)c->pdf[c->cur],
                                                                     (const C*)c->fb, a[0], a[1], a[2], rho, u);
    });
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_set_fb(es_ctx* c, const double* src) {
    c->fb_lazy = false;  // (the given field is used until the next solve)
    long long n = 3 * c->g.N;
    if (mixed(c))
        k_load_fb<float><<<blocks_for(n, 256), 256, 0, c->stream>>>(n, src, (float*)c->fb);
    else
        k_load_fb<double><<<blocks_for(n, 256), 256, 0, c->stream>>>(n, src, (double*)c->fb);
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_get_fb(es_ctx* c, double* dst) {
    const cudaError_t err = materialize_body_force(c);
    if (err != cudaSuccess) return err;
    long long n = 3 * c->g.N;
    if (mixed(c))
        k_copy_fb<float><<<blocks_for(n, 256), 256, 0, c->stream>>>(n, (const float*)c->fb, dst);
    else
        k_copy_fb<double><<<blocks_for(n, 256), 256, 0, c->stream>>>(n, (const double*)c->fb, dst);
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_gather(es_ctx* c, int which, const long long* idx, int n, double* out) {
    if (which == ES_FIELD_FB || which == ES_FIELD_U) {
        const cudaError_t err = materialize_body_force(c);
        if (err != cudaSuccess) return err;
    }
    const double* a = c->P.accel;
    int last = c->last_src >= 0 ? c->last_src : c->cur;
    dispatch_store(c, [&](auto tag) {
        using S = decltype(tag);
        using C = typename Store<S>::C;
        k_gather<S><<<blocks_for(n, 128), 128, 0, c->stream>>>(
            which, c->g.N, c->g.ps, idx, n, (const S*)c->pdf[c->cur], (const S*)c->pdf[last], (const C*)c->fb,
            c->psi, c->psi32, c->psi_lo, c->owner, c->flags, a[0], a[1], a[2], out);
    });
    count(c);
    return cudaGetLastError();
}

}  // namespace es
