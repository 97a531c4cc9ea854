// es_map.cu -- particle -> grid mapping, PDF reconstruction and potential
// stencil assembly (a1-a3; Sec. 4.2, Sec. 5.4, Sec. 5.5).
//
// The mapping follows the three-phase order of Sec. 5.5 so that spheres
// with overlapping bounding boxes never clobber each other: one kernel per
// phase, one thread block per sphere, threads striding over the sphere's
// bounding box only.
//   k_clear     cells owned by sphere p at the last mapping -> -2 - p
//   k_set       cells whose centre lies inside sphere p     -> p (atomicExch
//               detects a second claimant: overlap)
//   k_uncover   cells still marked -2 - p were uncovered: PDFs set to
//               f^eq(rho_0, u_s) of p's state at the last mapping
//   k_flags     flags / level-0 states of every cell within two cells of
//               the old or new sphere, and the count of p's fluid faces
//               (sigma = q / faces for a charged sphere)
#include "es_device.cuh"

namespace es {

namespace {

__global__ void k_init_flags(Grid g, uint8_t* flags, uint8_t* st0, int32_t* owner) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    long long c = lin(g, x, y, z);
    owner[c] = -1;
    bool near19 = false, near7 = false;
#pragma unroll
    for (int q = 1; q < 19; q++) {
        long long nb;
        if (!neighbour(g, x, y, z, cx(q), cy(q), cz(q), nb)) {
            near19 = true;
            if (q <= 3 || (q >= 10 && q <= 12)) near7 = true;
        }
    }
    flags[c] = near19 ? F_NEAR19 : 0;
    st0[c] = near7 ? ST_NEAR : ST_UNKNOWN;
}

struct Box {
    int lo[3], hi[3];
    __device__ int size(int a) const { return hi[a] - lo[a] + 1; }
    __device__ int count() const { return size(0) * size(1) * size(2); }
    // global coordinates of the cell with local index (i, j, k)
    __device__ __forceinline__ void at(const Grid& g, int i, int j, int k, int& x, int& y, int& z) const {
        x = wrap1(lo[0] + i, g.nx);
        y = wrap1(lo[1] + j, g.ny);
        z = wrap1(lo[2] + k, g.nz);
    }
    __device__ void cell(const Grid& g, int t, int& x, int& y, int& z) const {
        int sx = size(0), sy = size(1);
        int i = t % sx;
        int j = (t / sx) % sy;
        int k = t / (sx * sy);
        x = wrap_coord(lo[0] + i, g.nx);
        y = wrap_coord(lo[1] + j, g.ny);
        z = wrap_coord(lo[2] + k, g.nz);
    }
};

__device__ Box sphere_box(const Grid& g, const double* X, double R, int ext) {
    Box b;
    for (int a = 0; a < 3; a++) axis_range(g, a, X[a], X[a], R, ext, b.lo[a], b.hi[a]);
    return b;
}

// Union box of the old and the new position; on periodic axes the new
// position is taken as the image nearest to the old one.
__device__ Box union_box(const Grid& g, const double* Xo, const double* Xn, double R, int ext) {
    Box b;
    for (int a = 0; a < 3; a++) {
        double xo = Xo[a], xn = Xn[a];
        if (g.per[a]) {
            double L = (double)gdim(g, a);
            if (xn - xo > 0.5 * L) xn -= L;
            if (xn - xo < -0.5 * L) xn += L;
        }
        axis_range(g, a, fmin(xo, xn), fmax(xo, xn), R, ext, b.lo[a], b.hi[a]);
    }
    return b;
}

// GB300 runs FP64 arithmetic at a small fraction of the FP32 rate, so the
// per-sphere kernels form their FP64 set-up (box, FP32 ball) once per block
// in thread 0 and share it; per cell they work in integers and FP32 and
// fall back to the FP64 cell-in-sphere test only where FP32 cannot decide.

// Cells whose state flipped since the last solve (obstacle <-> fluid) go to
// a short list for the patched residual at the next solve's start
// (k_flip_patch); when it is full the next solve forms the residual in full.
struct FlipList {
    int* cells;
    int* count;
    int cap;
    int* full;  // set when a cell did not fit
    __device__ __forceinline__ void add(long long c) const {
        const int i = atomicAdd(count, 1);
        if (i < cap)
            cells[i] = (int)c;
        else
            *full = 1;
    }
};

__global__ void k_clear(Grid g, const DParticle* part, const double* mapped, int32_t* owner) {
    __shared__ Box sb;
    int p = blockIdx.x;
    if (threadIdx.x == 0) sb = sphere_box(g, mapped + 9 * p, part[p].R, 0);
    __syncthreads();
    const Box b = sb;
    int n = b.count();
    BoxWalk w;
    w.start(threadIdx.x, blockDim.x, b.size(0), b.size(1));
    for (int t = threadIdx.x; t < n; t += blockDim.x, w.next()) {
        int x, y, z;
        b.at(g, w.i, w.j, w.k, x, y, z);
        long long c = lin(g, x, y, z);
        if (owner[c] == p) owner[c] = -2 - p;
    }
}

__global__ void k_set(Grid g, const DParticle* part, const int* kind, int32_t* owner, double* psi,
                      float* psi_hi, float* psi_lo, int* status, FlipList flips) {
    __shared__ Box sb;
    __shared__ BallF sball;
    __shared__ double sbval;
    __shared__ float sbhi, sblo;
    int p = blockIdx.x;
    const DParticle& P = part[p];
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; a++)
            if (!g.per[a] && (P.x[a] - P.R < 0.0 || P.x[a] + P.R > (double)gdim(g, a)))
                atomicOr(status, DS_WALLCUT);
        // boundary value kept in the solution field at boundary cells (Sec. 5.4)
        sbval = kind[p] == ES_KIND_ZETA ? P.zeta : 0.0;
        const ff bff = ff_from_double(sbval);
        sbhi = bff.hi;
        sblo = bff.lo;
        sb = sphere_box(g, P.x, P.R, 0);
        sball.init(g, P.x, P.R, sb.lo, sb.hi);
    }
    __syncthreads();
    const Box b = sb;
    const BallF ball = sball;
    int n = b.count();
    BoxWalk w;
    w.start(threadIdx.x, blockDim.x, b.size(0), b.size(1));
    for (int t = threadIdx.x; t < n; t += blockDim.x, w.next()) {
        // decided in FP32 away from the surface, by the FP64 test near it
        int in = -1;
        if (ball.ok) {
            const float d2 = ball.d2(w.i, w.j, w.k);
            if (d2 > ball.r2 + ball.margin) continue;
            if (d2 < ball.r2 - ball.margin) in = 1;
        }
        int x, y, z;
        b.at(g, w.i, w.j, w.k, x, y, z);
        if (in < 0 && !cell_inside(g, P, x, y, z)) continue;
        long long c = lin(g, x, y, z);
        int old = atomicExch(&owner[c], p);
        if (old >= 0 && old != p) atomicOr(status, DS_OVERLAP);
        if (old == -1) flips.add(c);  // (a fluid cell became an obstacle cell)
        if (psi) {
            psi[c] = sbval;
        } else {
            psi_hi[c] = sbhi;
            psi_lo[c] = sblo;
        }
    }
}

template <class S>
__global__ void k_uncover(Grid g, const DParticle* part, const double* mapped, int32_t* owner, S* pdf,
                          FlipList flips) {
    __shared__ Box sb;
    int p = blockIdx.x;
    const double* M = mapped + 9 * p;  // x, v, w at the last mapping
    if (threadIdx.x == 0) sb = sphere_box(g, M, part[p].R, 0);
    __syncthreads();
    const Box b = sb;
    int n = b.count();
    BoxWalk w;
    w.start(threadIdx.x, blockDim.x, b.size(0), b.size(1));
    for (int t = threadIdx.x; t < n; t += blockDim.x, w.next()) {
        int x, y, z;
        b.at(g, w.i, w.j, w.k, x, y, z);
        long long c = lin(g, x, y, z);
        if (owner[c] != -2 - p) continue;
        owner[c] = -1;
        flips.add(c);  // (an obstacle cell became a fluid cell)
        double u[3];
        surface_velocity(g, M, M + 3, M + 6, x, y, z, u);
        double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
        for (int q = 0; q < 19; q++) {
            double cu = cx(q) * u[0] + cy(q) * u[1] + cz(q) * u[2];
            // f^eq(rho_0 = 1, u_s) of Eq. fequ_Incompr_SRT
            double dev = wq(q) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            pdf[(long long)q * g.ps + c] = Store<S>::from_dev(q, dev);
        }
    }
}

// Flags of one cell from the owner field.  Returns the number of D3Q7 faces
// the cell (if fluid) shares with sphere `p`.
__device__ int cell_flags(const Grid& g, const int32_t* owner, const int* kind, int x, int y, int z,
                          int p, uint8_t& fl, uint8_t& st) {
    long long c = lin(g, x, y, z);
    int o = owner[c];
    if (o >= 0) {
        fl = F_SOLID;
        st = kind[o] == ES_KIND_ZETA ? ST_DIR : ST_NEU;
        return 0;
    }
    bool near19 = false, near7 = false;
    int faces = 0;
#pragma unroll
    for (int q = 1; q < 19; q++) {
        long long nb;
        bool axis = (q <= 3) || (q >= 10 && q <= 12);
        if (!neighbour(g, x, y, z, cx(q), cy(q), cz(q), nb)) {
            near19 = true;
            near7 |= axis;
            continue;
        }
        int on = owner[nb];
        if (on >= 0) {
            near19 = true;
            near7 |= axis;
            if (axis && on == p) faces++;
        }
    }
    fl = near19 ? F_NEAR19 : 0;
    st = near7 ? ST_NEAR : ST_UNKNOWN;
    return faces;
}

// all_cells = 0 skips the cells whose flags cannot have changed.  With D
// the displacement since the last mapping, a cell that changed owner lies
// within D of the old surface in its old distance and within D of the new
// surface in its new distance; a cell whose D3Q19 neighbours (within
// sqrt 2) include one is therefore within D + sqrt 2 of both.  A cell
// outside either band keeps its flags, and it has no D3Q7 face to the new
// sphere unless it is within 1 of the new surface.  So a cell is visited
// when it is within 2.5 of the new surface, or within 2.5 + D of both.
// The first mapping of a context visits every cell (all_cells = 1).
__global__ void k_flags(Grid g, DParticle* part, const double* mapped, const int* kind,
                        const int32_t* owner, uint8_t* flags, uint8_t* st0, int* nfaces, int all_cells) {
    __shared__ int tile[kOwnerTileMax];
    __shared__ Box sb;
    __shared__ BallF sbo, sbn;
    __shared__ float sband[5];  // lo1, hi1, lo2, hi2, skip_ok
    __shared__ int sw[32];
    int p = blockIdx.x;
    if (threadIdx.x == 0) {
        const double* Xo = mapped + 9 * p;
        const double R = part[p].R;
        sb = union_box(g, Xo, part[p].x, R, 2);
        sbo.init(g, Xo, R, sb.lo, sb.hi);
        sbn.init(g, part[p].x, R, sb.lo, sb.hi);
        float D2 = 0.0f;
        for (int a = 0; a < 3; a++) {
            double d = part[p].x[a] - Xo[a];
            if (g.per[a]) {
                const double L = (double)gdim(g, a);
                if (d > 0.5 * L) d -= L;
                if (d < -0.5 * L) d += L;
            }
            D2 += (float)d * (float)d;
        }
        // (bands: faces need the new surface's outer layer, R .. R + 1;
        // changed flags lie within sqrt 2 + D of both surfaces; 0.05 margin)
        const float rf = (float)R, w1 = 1.05f, w2 = 1.47f + sqrtf(D2) * 1.001f;
        sband[0] = rf > w1 ? (rf - w1) * (rf - w1) : -1.0f;
        sband[1] = (rf + w1) * (rf + w1);
        sband[2] = rf > w2 ? (rf - w2) * (rf - w2) : -1.0f;
        sband[3] = (rf + w2) * (rf + w2);
        sband[4] = (!all_cells && sbo.ok && sbn.ok) ? 1.0f : 0.0f;
    }
    __syncthreads();
    const Box b = sb;
    const BallF bo = sbo, bn = sbn;
    const float lo1 = sband[0], hi1 = sband[1], lo2 = sband[2], hi2 = sband[3];
    const bool skip_ok = sband[4] != 0.0f;
    const OwnerTile T{{b.size(0), b.size(1), b.size(2)}};
    const bool use_tile = T.fits();
    if (use_tile) {
        load_owner_tile(g, owner, b.lo, T, tile);
        __syncthreads();
    }
    int n = b.count();
    int faces = 0;
    BoxWalk w;
    w.start(threadIdx.x, blockDim.x, b.size(0), b.size(1));
    for (int t = threadIdx.x; t < n; t += blockDim.x, w.next()) {
        if (skip_ok) {
            const float dn = bn.d2(w.i, w.j, w.k), dol = bo.d2(w.i, w.j, w.k);
            const bool near_new = dn >= lo1 && dn <= hi1;
            const bool near_both = dn >= lo2 && dn <= hi2 && dol >= lo2 && dol <= hi2;
            if (!near_new && !near_both) continue;
        }
        int x, y, z;
        b.at(g, w.i, w.j, w.k, x, y, z);
        uint8_t fl, st;
        if (use_tile) {
            // cell_flags from the tile
            const int ti = T.at(w.i, w.j, w.k);
            const int o = tile[ti];
            if (o >= 0) {
                fl = F_SOLID;
                st = kind[o] == ES_KIND_ZETA ? ST_DIR : ST_NEU;
            } else {
                bool near19 = false, near7 = false;
#pragma unroll
                for (int q = 1; q < 19; q++) {
                    const int on = tile[ti + T.step(q)];
                    const bool axis = (q <= 3) || (q >= 10 && q <= 12);
                    if (on >= 0 || on == kOwnerOutside) {
                        near19 = true;
                        near7 |= axis;
                        if (axis && on == p) faces++;
                    }
                }
                fl = near19 ? F_NEAR19 : 0;
                st = near7 ? ST_NEAR : ST_UNKNOWN;
            }
        } else {
            faces += cell_flags(g, owner, kind, x, y, z, p, fl, st);
        }
        long long c = lin(g, x, y, z);
        flags[c] = fl;
        st0[c] = st;
    }
    // block sum of the face counts (integers: exact in any order)
    for (int o = 16; o > 0; o >>= 1) faces += __shfl_down_sync(0xffffffffu, faces, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = faces;
    __syncthreads();
    if (threadIdx.x == 0) {
        int nf = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) nf += sw[w];
        nfaces[p] = nf;
        // Neumann charge per face: sigma = q / faces, so that the flux over
        // the staircase surface equals the particle charge.
        part[p].sigma = nf > 0 ? part[p].q / (double)nf : 0.0;
    }
}

// Keeps the mapped state for the next reconstruction and, in the MIXED32
// form, the sphere's boundary value for the float-float outer residual:
// 2 zeta for a Dirichlet sphere, sigma / eps for a charged one (Sec. 5.4).
// Raises *moved when the sphere moved half a cell or more along an axis
// since the previous mapping (minimum image on periodic axes).
__global__ void k_store_mapped(Grid g, const DParticle* part, const int* kind, double eps, double* mapped,
                               float* pbc, int np, int* moved) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    for (int a = 0; a < 3; a++) {
        double d = fabs(part[p].x[a] - mapped[9 * p + a]);
        const double L = (double)gdim(g, a);
        if (g.per[a] && d > 0.5 * L) d = L - d;
        if (!(d < 0.5)) *moved = 1;
    }
    for (int a = 0; a < 3; a++) {
        mapped[9 * p + a] = part[p].x[a];
        mapped[9 * p + 3 + a] = part[p].v[a];
        mapped[9 * p + 6 + a] = part[p].w[a];
    }
    if (pbc) {
        const ff v = ff_from_double(kind[p] == ES_KIND_ZETA ? 2.0 * part[p].zeta : part[p].sigma / eps);
        pbc[2 * p] = v.hi;
        pbc[2 * p + 1] = v.lo;
    }
}

// Coarse level states (multigrid design): Dirichlet if any child is
// Dirichlet, else unknown if any child is unknown, else Neumann.
__global__ void k_coarse_kind(int fx, int fy, int fz, int cxn, int cyn, int czn, const uint8_t* fine,
                              uint8_t* coarse) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y, k = blockIdx.z;
    if (i >= cxn) return;
    bool any_dir = false, any_unknown = false;
    for (int dk = 0; dk < 2; dk++)
        for (int dj = 0; dj < 2; dj++)
            for (int di = 0; di < 2; di++) {
                uint8_t s = fine[(long long)(2 * i + di) + (long long)fx * ((long long)(2 * j + dj) + (long long)fy * (2 * k + dk))] & ST_KIND;
                any_dir |= (s == ST_DIR);
                any_unknown |= (s == ST_UNKNOWN);
            }
    coarse[(long long)i + (long long)cxn * ((long long)j + (long long)cyn * k)] =
        any_dir ? ST_DIR : (any_unknown ? ST_UNKNOWN : ST_NEU);
    (void)fz;
    (void)czn;
}

// Coarse kinds, four coarse cells per thread (coarse nx % 4 == 0): the 8
// fine cells of a fine row segment arrive as one 8-byte load per child row.
__global__ void __launch_bounds__(256) k_coarse_kind_v(int fx, int fy, int cxn, int cyn,
                                                       const uint8_t* __restrict__ fine,
                                                       uint8_t* __restrict__ coarse) {
    const int i0 = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i0 >= cxn || j >= cyn) return;
    unsigned any_dir = 0, any_unk = 0;  // bit per coarse cell
#pragma unroll
    for (int dk = 0; dk < 2; dk++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++) {
            const uint2 v = *reinterpret_cast<const uint2*>(
                fine + (size_t)2 * i0 + (size_t)fx * ((size_t)(2 * j + dj) + (size_t)fy * (2 * k + dk)));
#pragma unroll
            for (int b = 0; b < 8; b++) {
                const unsigned s = ((b < 4 ? v.x : v.y) >> (8 * (b & 3))) & ST_KIND;
                if (s == ST_DIR) any_dir |= 1u << (b >> 1);
                if (s == ST_UNKNOWN) any_unk |= 1u << (b >> 1);
            }
        }
    unsigned out = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const unsigned kind = ((any_dir >> q) & 1u) ? ST_DIR : (((any_unk >> q) & 1u) ? ST_UNKNOWN : ST_NEU);
        out |= kind << (8 * q);
    }
    *reinterpret_cast<unsigned*>(coarse + (size_t)i0 + (size_t)cxn * ((size_t)j + (size_t)cyn * k)) = out;
}

// Near-boundary bits of a level (as k_near_bits), four cells per thread
// (nx % 4 == 0), in place: a thread rewrites its 4-byte word with the same
// kind bits, and neighbours read only kind bits, so every read sees the
// kinds whether or not the word was rewritten yet.
__global__ void __launch_bounds__(256) k_near_bits_v(int nx, int ny, int nz, int px, int py, int pz, uint8_t* st) {
    const int i0 = 4 * (blockIdx.x * 32 + threadIdx.x);
    const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i0 >= nx || j >= ny) return;
    const size_t row = (size_t)nx * ((size_t)j + (size_t)ny * k);
    const unsigned own = *reinterpret_cast<const unsigned*>(st + row + i0);
    // the kinds of the four neighbour rows at the same x, and the x halo
    // (a missing neighbour beyond a wall counts as not unknown)
    const unsigned kOut = 0x02020202u;  // (Neumann: not unknown)
    auto row_at = [&](int jj, int kk) -> unsigned {
        return *reinterpret_cast<const unsigned*>(st + (size_t)nx * ((size_t)jj + (size_t)ny * kk) + i0);
    };
    unsigned ym = kOut, yp = kOut, zm = kOut, zp = kOut;
    if (j > 0) ym = row_at(j - 1, k); else if (py) ym = row_at(ny - 1, k);
    if (j < ny - 1) yp = row_at(j + 1, k); else if (py) yp = row_at(0, k);
    if (k > 0) zm = row_at(j, k - 1); else if (pz) zm = row_at(j, nz - 1);
    if (k < nz - 1) zp = row_at(j, k + 1); else if (pz) zp = row_at(j, 0);
    unsigned xl = 2u, xr = 2u;
    if (i0 > 0) xl = st[row + i0 - 1]; else if (px) xl = st[row + nx - 1];
    if (i0 + 4 < nx) xr = st[row + i0 + 4]; else if (px) xr = st[row];
    unsigned res = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const unsigned s = (own >> (8 * q)) & ST_KIND;
        unsigned v = s;
        if (s == ST_UNKNOWN) {
            const unsigned l = q == 0 ? (xl & ST_KIND) : ((own >> (8 * (q - 1))) & ST_KIND);
            const unsigned r = q == 3 ? (xr & ST_KIND) : ((own >> (8 * (q + 1))) & ST_KIND);
            const bool near = l != ST_UNKNOWN || r != ST_UNKNOWN || ((ym >> (8 * q)) & ST_KIND) != ST_UNKNOWN ||
                              ((yp >> (8 * q)) & ST_KIND) != ST_UNKNOWN ||
                              ((zm >> (8 * q)) & ST_KIND) != ST_UNKNOWN ||
                              ((zp >> (8 * q)) & ST_KIND) != ST_UNKNOWN;
            v = near ? (ST_UNKNOWN | ST_NEAR) : ST_UNKNOWN;
        }
        res |= v << (8 * q);
    }
    *reinterpret_cast<unsigned*>(st + row + i0) = res;
}

// Near-boundary bit of an unknown cell: a D3Q7 neighbour that is not an
// unknown, or a non-periodic domain face.  Only the bit is written; the
// kind bits neighbours read are unchanged, so updating in place is safe.
__global__ void k_near_bits(int nx, int ny, int nz, int px, int py, int pz, uint8_t* st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    long long c = (long long)i + (long long)nx * ((long long)j + (long long)ny * k);
    uint8_t s = st[c];
    if ((s & ST_KIND) != ST_UNKNOWN) return;
    bool near = false;
    int n3[3] = {nx, ny, nz}, p3[3] = {px, py, pz}, v[3] = {i, j, k};
    for (int a = 0; a < 3 && !near; a++)
        for (int d = -1; d <= 1 && !near; d += 2) {
            int w = v[a] + d;
            if (w < 0 || w >= n3[a]) {
                if (!p3[a]) {
                    near = true;
                    break;
                }
                w = w < 0 ? w + n3[a] : w - n3[a];
            }
            int q[3] = {v[0], v[1], v[2]};
            q[a] = w;
            uint8_t t = st[(long long)q[0] + (long long)nx * ((long long)q[1] + (long long)ny * q[2])] & ST_KIND;
            if (t != ST_UNKNOWN) near = true;
        }
    st[c] = near ? (uint8_t)(ST_UNKNOWN | ST_NEAR) : (uint8_t)ST_UNKNOWN;
}

// Exclusive prefix sum of v over the warp; total = the sum of all lanes.
__device__ __forceinline__ int warp_excl_scan(int v, int& total) {
    const int lane = threadIdx.x & 31;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - v;
}

// Lists the near-boundary unknown cells of a level, by colour, for the
// separate near-cell passes of the smoother, residual and restriction.  A
// row (y, z) goes to segment row mod kNearSegs of each colour; a warp walks
// its row 256 cells at a time, lane l taking cells l, l + 32, ..., which
// all have one colour, with one prefix sum and one atomic per colour on the
// segment's counters.  The order within a segment depends on the atomics'
// order; the consumers write each cell's value to its own place, so results
// do not.  With rbmask (a colour-split level, nx even), also its per-colour
// update masks as k_lists_l0 builds them: a 32-cell step holds 16 cells of
// each colour, compact places x0 / 2 .. x0 / 2 + 15, which fill the low or
// the high half of one word.
__global__ void __launch_bounds__(256) k_near_list(int nx, int ny, int nz, const uint8_t* __restrict__ st,
                                                   int cap, int* list, int* count, uint32_t* __restrict__ rbmask,
                                                   int wpr) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= ny * nz) return;  // whole warps
    const int seg = row % kNearSegs;
    const int y = row % ny, z = row / ny;
    const int colour = (lane + y + z) & 1;  // of the lane's cells (steps of 32 keep it)
    unsigned pend[2] = {0u, 0u};  // (low halves of the mask words, stored with their high halves)
    for (int xb = 0; xb < nx; xb += 8 * 32) {
        // the state bytes of eight 32-cell steps, all loaded before the
        // first is tested, so that a warp has eight loads in flight
        uint8_t sv[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int x = xb + 32 * q + lane;
            sv[q] = x < nx ? st[x + nx * row] : (uint8_t)0;
        }
        unsigned tk = 0;  // bit q: cell xb + 32 q + lane is listed
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int x0 = xb + 32 * q;
            if (x0 >= nx) break;  // (warp-uniform)
            const int x = x0 + lane;
            bool take = false, inner = false;
            if (x < nx) {
                const uint8_t s = sv[q];
                take = (s & ST_KIND) == ST_UNKNOWN && (s & ST_NEAR);
                inner = (s & (ST_KIND | ST_NEAR)) == ST_UNKNOWN;
            }
            tk |= (take ? 1u : 0u) << q;
            if (rbmask) {
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    const bool b = inner && colour == k;
                    const unsigned v = __reduce_or_sync(0xffffffffu, b ? 1u << (lane >> 1) : 0u);
                    const bool last = x0 + 32 >= nx;
                    if ((x0 & 63) == 0) pend[k] = v;
                    if (lane == 0 && ((x0 & 63) != 0 || last)) {
                        // the word of compact places x0/2 & ~31 .. +31 (a high half past the row's end stays 0)
                        const unsigned word = (x0 & 63) != 0 ? (pend[k] | (v << 16)) : v;
                        rbmask[(size_t)k * ((size_t)ny * nz * wpr) + (size_t)wpr * row + x0 / 64] = word;
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, tk != 0)) continue;
        // one scan for both colours, in 10-bit fields (at most 128 cells of
        // a colour in 256)
        int total;
        const int excl = warp_excl_scan(__popc(tk) << (10 * colour), total);
        int base = 0;
        if (lane < 2) {
            const int tl = (total >> (10 * lane)) & 0x3FF;
            if (tl) base = atomicAdd(&count[lane * kNearSegs + seg], tl);
        }
        const int b0 = __shfl_sync(0xffffffffu, base, 0), b1 = __shfl_sync(0xffffffffu, base, 1);
        int k = (colour ? b1 : b0) + ((excl >> (10 * colour)) & 0x3FF);
        int* out = list + (size_t)(colour * kNearSegs + seg) * cap;
        for (unsigned m = tk; m; m &= m - 1u) {
            const int q = __ffs(m) - 1;
            if (k < cap) out[k] = xb + 32 * q + lane + nx * row;
            k++;
        }
    }
}

// Lists the fluid cells with a non-fluid D3Q19 neighbour (F_NEAR19), which
// the body force treats with the D3Q7 ghost-value gradient, in kNearSegs
// row segments as k_near_list does.
__global__ void __launch_bounds__(256) k_near19_list(int nx, int ny, int nz, const uint8_t* __restrict__ flags,
                                                     int cap, int* list, int* count) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= ny * nz) return;  // whole warps
    const int seg = row % kNearSegs;
    for (int x0 = 0; x0 < nx; x0 += 32) {
        const int x = x0 + lane;
        bool take = false;
        if (x < nx) {
            const uint8_t f = flags[x + nx * row];
            take = (f & F_NEAR19) && !(f & F_SOLID);
        }
        const unsigned m = __ballot_sync(0xffffffffu, take);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&count[seg], __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (take) {
            const int i = base + __popc(m & lt);
            if (i < cap) list[(size_t)seg * cap + i] = x + nx * row;
        }
    }
}

// Level 0 in one pass: both lists (near-boundary unknown cells by colour,
// and fluid cells next to obstacles) from 4 cells per lane (x extent a
// multiple of 4), a warp per row, 512 cells at a time.  The counts of the
// chunk's four 128-cell spans go through one warp prefix sum and one atomic
// per list, so that a warp waits for one atomic round trip per chunk.
// With rbmask (the colour-split finest level), also the per-colour update
// masks of the half sweeps: bit j of colour k's row (wpr words, compact
// index j = x / 2) is set iff that cell is an interior unknown cell.
__global__ void __launch_bounds__(256) k_lists_l0(int nx, int ny, int nz, const uint8_t* __restrict__ st,
                                                  const uint8_t* __restrict__ flags, int cap, int* list,
                                                  int* count, int bf_cap, int* bf_list, int* bf_count,
                                                  uint32_t* __restrict__ rbmask, int wpr) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= ny * nz) return;  // whole warps
    const int seg = row % kNearSegs;
    const int y = row % ny, z = row / ny;
    const int p0 = (y + z) & 1;  // colour of the cells x with x % 4 = 0 or 2
    auto nibble = [](unsigned b) { return ((b & 0x01010101u) * 0x01020408u) >> 24; };
    for (int xb = 0; xb < nx; xb += 4 * 128) {
        // the words of four 128-cell spans, all loaded before the first is
        // tested, so that a warp has eight loads in flight
        unsigned swv[4], fwv[4];
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const int xs = xb + 128 * s + 4 * lane;
            swv[s] = 0x02020202u;  // (Neumann / obstacle: not listed)
            fwv[s] = 0x01010101u;
            if (xs < nx) {
                swv[s] = *reinterpret_cast<const unsigned*>(st + xs + nx * row);
                fwv[s] = *reinterpret_cast<const unsigned*>(flags + xs + nx * row);
            }
        }
        // the lane's listed cells: bit 4 s + i of ms[t] is cell
        // xb + 128 s + 4 lane + i of list t (near cells of colour p0, of the
        // other colour, fluid cells next to obstacles)
        unsigned ms[3] = {0u, 0u, 0u};
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const int x0 = xb + 128 * s;
            if (x0 >= nx) break;  // (warp-uniform)
            // the three tests on the lane's four cells at once: bit 0 of each
            // byte (state values < 8, flag values < 4) gathered into a nibble,
            // cell i at bit i
            const unsigned sw = swv[s] & 0x07070707u, fw = fwv[s] & 0x03030303u;
            const unsigned in4 = nibble(~(sw | (sw >> 1) | (sw >> 2)));  // state 0: interior unknown cell
            const unsigned nr4 = nibble((sw >> 2) & ~(sw | (sw >> 1)));  // state 4: near-boundary unknown cell
            const unsigned bf4 = nibble((fw >> 1) & ~fw);                // flags 2: next to an obstacle, fluid
            if (rbmask) {
                // lane's cells of colour k: x0 + 4 lane + O and + 2 + O,
                // O = k ^ p0, at compact places 2 lane and 2 lane + 1 of
                // this span's 64
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    const int O = k ^ p0;
                    const unsigned v = ((in4 >> O) & 1u) | (((in4 >> (O + 2)) & 1u) << 1);
                    const unsigned sh = v << ((2 * lane) & 31);
                    const unsigned lo = __reduce_or_sync(0xffffffffu, lane < 16 ? sh : 0u);
                    const unsigned hi = __reduce_or_sync(0xffffffffu, lane < 16 ? 0u : sh);
                    const int w0 = x0 / 64;  // (x0 is a multiple of 128)
                    uint32_t* m = rbmask + (size_t)k * ((size_t)ny * nz * wpr) + (size_t)wpr * row;
                    if (lane == 0) m[w0] = lo;
                    if (lane == 16 && w0 + 1 < wpr) m[w0 + 1] = hi;
                }
            }
            // near-boundary cells by colour: cells i = 0, 2 have colour p0, i = 1, 3 the other
            ms[0] |= (nr4 & 0x5u) << (4 * s);
            ms[1] |= (nr4 & 0xAu) << (4 * s);
            ms[2] |= bf4 << (4 * s);
        }
        // (most chunks hold no listed cell: one vote skips them)
        if (!__any_sync(0xffffffffu, (ms[0] | ms[1] | ms[2]) != 0)) continue;
        // one scan for the three lists, in fields of 10, 10 and 11 bits (a
        // warp lists at most 256 cells of a colour and 512 next to obstacles)
        int total;
        const int excl =
            warp_excl_scan((int)(__popc(ms[0]) | (__popc(ms[1]) << 10) | (__popc(ms[2]) << 20)), total);
        int base = 0;
        if (lane < 3) {
            const int tl = (total >> (10 * lane)) & (lane < 2 ? 0x3FF : 0x7FF);
            // (ms[t] holds cells of colour t ^ p0)
            int* cnt = lane < 2 ? &count[(lane ^ p0) * kNearSegs + seg] : &bf_count[seg];
            if (tl) base = atomicAdd(cnt, tl);
        }
#pragma unroll
        for (int t = 0; t < 3; t++) {
            const int bt = __shfl_sync(0xffffffffu, base, t);
            const int kl = t < 2 ? t ^ p0 : 2;  // (list 0, 1: colour; 2: next to obstacles)
            int* out = kl < 2 ? list + (size_t)(kl * kNearSegs + seg) * cap : bf_list + (size_t)seg * bf_cap;
            const int c_out = kl < 2 ? cap : bf_cap;
            int k = bt + ((excl >> (10 * t)) & (t < 2 ? 0x3FF : 0x7FF));
            for (unsigned m = ms[t]; m; m &= m - 1u) {
                const int b = __ffs(m) - 1;
                if (k < c_out) out[k] = xb + 128 * (b >> 2) + 4 * lane + (b & 3) + nx * row;
                k++;
            }
        }
    }
}

}  // namespace

cudaError_t launch_near_lists(es_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->near_count, 0, 2 * kNearSegs * ES_MAXLEV * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c->bf_count, 0, kNearSegs * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    int l0 = 0;
    if (c->g.nx % 4 == 0) {
        ProfScope ps(c, "cell_lists", 0, 2.0 * (double)c->g.N);
        k_lists_l0<<<(c->g.ny * c->g.nz + 7) / 8, 256, 0, c->stream>>>(c->g.nx, c->g.ny, c->g.nz, c->st[0], c->flags,
                                                                      c->near_cap[0], c->near_list[0], c->near_count,
                                                                      c->bf_cap, c->bf_list, c->bf_count,
                                                                      c->rbmask, c->rb_wpr);
        count(c);
        l0 = 1;
    }
    for (int l = l0; l < c->L; l++) {
        const int* n = c->ln[l];
        const int rows = n[1] * n[2];
        const int nb = (rows + 7) / 8;  // a warp per row: every row in flight at once
        ProfScope ps(c, "cell_lists", l, (double)rows * n[0]);
        k_near_list<<<nb, 256, 0, c->stream>>>(n[0], n[1], n[2], c->st[l], c->near_cap[l], c->near_list[l],
                                                c->near_count + 2 * kNearSegs * l, l == 1 ? c->rbmask1 : nullptr,
                                                c->rb_wpr1);
        count(c);
    }
    if (l0 == 0) {
        k_near19_list<<<(c->g.ny * c->g.nz + 7) / 8, 256, 0, c->stream>>>(c->g.nx, c->g.ny, c->g.nz, c->flags,
                                                                          c->bf_cap, c->bf_list, c->bf_count);
        count(c);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_flags(es_ctx* c) {
    const Grid& g = c->g;
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny, g.nz);
    k_init_flags<<<grd, blk, 0, c->stream>>>(g, c->flags, c->st[0], c->owner);
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_map(es_ctx* c) {
    if (c->np == 0) return cudaSuccess;
    const Grid& g = c->g;
    const int T = 256;
    const FlipList flips{c->flip_list, c->flip_count, c->flip_cap, c->d_moved};
    {
        ProfScope ps(c, "map_clear", -1, 0.0);
        k_clear<<<c->np, T, 0, c->stream>>>(g, c->part, c->mapped, c->owner);
    }
    {
        ProfScope ps(c, "map_set", -1, 0.0);
        k_set<<<c->np, T, 0, c->stream>>>(g, c->part, c->kind, c->owner, c->psi, c->psi32, c->psi_lo, c->d_status,
                                          flips);
    }
    {
        ProfScope ps(c, "map_uncover", -1, 0.0);
        if (c->P.precision == ES_MIXED16)
            k_uncover<__half><<<c->np, T, 0, c->stream>>>(g, c->part, c->mapped, c->owner, (__half*)c->pdf[c->cur],
                                                            flips);
        else if (mixed(c))
            k_uncover<float><<<c->np, T, 0, c->stream>>>(g, c->part, c->mapped, c->owner, (float*)c->pdf[c->cur],
                                                           flips);
        else
            k_uncover<double><<<c->np, T, 0, c->stream>>>(g, c->part, c->mapped, c->owner, (double*)c->pdf[c->cur],
                                                            flips);
    }
    {
        ProfScope ps(c, "map_flags", -1, 0.0);
        k_flags<<<c->np, T, 0, c->stream>>>(g, c->part, c->mapped, c->kind, c->owner, c->flags, c->st[0],
                                            c->nfaces, c->mapped_once ? 0 : 1);
        c->mapped_once = true;
    }
    k_store_mapped<<<(c->np + 127) / 128, 128, 0, c->stream>>>(g, c->part, c->kind, c->S.eps, c->mapped, c->pbc,
                                                                c->np, c->d_moved);
    count(c, 5);
    return cudaGetLastError();
}

cudaError_t launch_coarse_states(es_ctx* c) {
    for (int l = 1; l < c->L; l++) {
        const int* f = c->ln[l - 1];
        const int* m = c->ln[l];
        dim3 blk(128), grd((m[0] + 127) / 128, m[1], m[2]);
        const double nc = (double)m[0] * m[1] * m[2];
        ProfScope ps(c, "coarse_states", l, 8.0 * nc + nc + 2.0 * nc);
        if (m[0] % 4 == 0) {
            const dim3 vblk(32, 8), vgrd((m[0] / 4 + 31) / 32, (m[1] + 7) / 8, m[2]);
            k_coarse_kind_v<<<vgrd, vblk, 0, c->stream>>>(f[0], f[1], m[0], m[1], c->st[l - 1], c->st[l]);
            k_near_bits_v<<<vgrd, vblk, 0, c->stream>>>(m[0], m[1], m[2], c->g.per[0], c->g.per[1], c->g.per[2],
                                                         c->st[l]);
        } else {
            k_coarse_kind<<<grd, blk, 0, c->stream>>>(f[0], f[1], f[2], m[0], m[1], m[2], c->st[l - 1], c->st[l]);
            k_near_bits<<<grd, blk, 0, c->stream>>>(m[0], m[1], m[2], c->g.per[0], c->g.per[1], c->g.per[2],
                                                    c->st[l]);
        }
        count(c, 2);
    }
    return cudaGetLastError();
}

}  // namespace es
