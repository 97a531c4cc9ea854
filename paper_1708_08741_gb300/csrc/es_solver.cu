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
// The outer loop runs in FP64 on psi; the V-cycle solves A e = r for the
// correction in the inner type T (double, or float in the MIXED32 form).
#include "es_device.cuh"

namespace es {

namespace {

constexpr int kRedThreads = 256;

struct LevelDesc {
    int nx, ny, nz;
    int per[3];
    int pot_bc[6];
    double h2;    // h_l^2
    double diag0; // 6 + kappa^2 h_l^2
};

// Fine-level face contribution for the FP64 outer residual: adds the centre
// adjustment to diag and the boundary value to b, or returns the neighbour
// index of an unknown neighbour (>= 0).
__device__ __forceinline__ long long fine_face(const Grid& g, const Solver& s, const int32_t* owner,
                                               const DParticle* part, const int* kind, int x, int y,
                                               int z, int a, int side, double& diag, double& b) {
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
    if (o < 0) return nb;
    if (kind[o] == ES_KIND_ZETA) {
        diag += 1.0;
        b += 2.0 * part[o].zeta;
    } else {
        diag -= 1.0;
        b += part[o].sigma / s.eps;
    }
    return -1;
}

// r = b - A psi on the unknowns (FP64), stored as the V-cycle right-hand
// side in type T, and per-block partial sums of r^2.
template <class T>
__global__ void __launch_bounds__(kRedThreads) k_outer_residual(Grid g, Solver s, const double* psi,
                                                                const uint8_t* st0, const int32_t* owner,
                                                                const DParticle* part, const int* kind,
                                                                T* r_out, double* partial) {
    __shared__ double sh[32];
    double acc = 0.0;
    const double diag0 = 6.0 + s.kappa * s.kappa;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < g.N; c += stride) {
        uint8_t st = st0[c];
        double r = 0.0;
        if ((st & ST_KIND) == ST_UNKNOWN) {
            int x = (int)(c % g.nx);
            long long yz = c / g.nx;
            int y = (int)(yz % g.ny);
            int z = (int)(yz / g.ny);
            double diag = diag0, b = 0.0, off = 0.0;
            if (!(st & ST_NEAR)) {
                int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
                int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
                int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
                off = psi[lin(g, xm, y, z)];
                off += psi[lin(g, xp, y, z)];
                off += psi[lin(g, x, ym, z)];
                off += psi[lin(g, x, yp, z)];
                off += psi[lin(g, x, y, zm)];
                off += psi[lin(g, x, y, zp)];
            } else {
                for (int a = 0; a < 3; a++)
                    for (int side = -1; side <= 1; side += 2) {
                        long long nb = fine_face(g, s, owner, part, kind, x, y, z, a, side, diag, b);
                        if (nb >= 0) off += psi[nb];
                    }
            }
            r = b - (diag * psi[c] - off);
            acc += r * r;
        }
        r_out[c] = (T)r;
    }
    double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_finalize_norm(const double* partial, int n, double* out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
    double tot = block_sum(v, sh);
    if (threadIdx.x == 0) out[0] = sqrt(tot);
}

// Diagonal and off-diagonal sum of level l at an unknown cell.  With
// READ = false only the diagonal is formed (off = 0, e is not touched).
template <class T, bool READ = true>
__device__ __forceinline__ void level_stencil(const LevelDesc& L, const uint8_t* st, const T* e, int x,
                                              int y, int z, uint8_t s, T& diag, T& off) {
    long long nxny = (long long)L.nx * L.ny;
    if (!READ && !(s & ST_NEAR)) {
        diag = (T)L.diag0;
        off = (T)0;
        return;
    }
    if (!(s & ST_NEAR)) {
        int xm = x == 0 ? L.nx - 1 : x - 1, xp = x == L.nx - 1 ? 0 : x + 1;
        int ym = y == 0 ? L.ny - 1 : y - 1, yp = y == L.ny - 1 ? 0 : y + 1;
        int zm = z == 0 ? L.nz - 1 : z - 1, zp = z == L.nz - 1 ? 0 : z + 1;
        long long row = (long long)y * L.nx + (long long)z * nxny;
        off = e[row + xm];
        off += e[row + xp];
        off += e[(long long)ym * L.nx + (long long)z * nxny + x];
        off += e[(long long)yp * L.nx + (long long)z * nxny + x];
        off += e[(long long)y * L.nx + (long long)zm * nxny + x];
        off += e[(long long)y * L.nx + (long long)zp * nxny + x];
        diag = (T)L.diag0;
        return;
    }
    double dg = L.diag0;
    T o = (T)0;
    int v[3] = {x, y, z}, n3[3] = {L.nx, L.ny, L.nz};
    for (int a = 0; a < 3; a++)
        for (int side = -1; side <= 1; side += 2) {
            int w[3] = {v[0], v[1], v[2]};
            int p = v[a] + side;
            if (p < 0 || p >= n3[a]) {
                if (!L.per[a]) {
                    dg += (L.pot_bc[2 * a + (side > 0 ? 1 : 0)] == ES_POT_DIRICHLET) ? 1.0 : -1.0;
                    continue;
                }
                p = p < 0 ? p + n3[a] : p - n3[a];
            }
            w[a] = p;
            long long nb = (long long)w[0] + (long long)L.nx * w[1] + nxny * w[2];
            uint8_t k = st[nb] & ST_KIND;
            if (k == ST_UNKNOWN) {
                if (READ) o += e[nb];
            }
            else
                dg += (k == ST_DIR) ? 1.0 : -1.0;
        }
    diag = (T)dg;
    off = o;
}

// One red (colour 0) or black (1) Gauss-Seidel / SOR half sweep,
// colour = (i + j + k) mod 2.  Thread t owns the cell pair (2t, 2t+1) of a
// row and updates the one of this colour.  first != 0: the iterate starts
// at zero, so neighbours are not read and the pair's other cell is zeroed.
template <class T>
__global__ void __launch_bounds__(128) k_smooth(LevelDesc L, const uint8_t* st, const T* rhs, T* e,
                                                int colour, int first, T omega) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    if (2 * t >= L.nx) return;
    int par = (colour + y + z) & 1;
    int x = 2 * t + par;
    long long row = (long long)L.nx * ((long long)y + (long long)L.ny * z);
    if (first && 2 * t + 1 - par < L.nx) e[row + 2 * t + 1 - par] = (T)0;
    if (x >= L.nx) return;  // odd extent: the last pair has one cell
    long long c = row + x;
    uint8_t s = st[c];
    if ((s & ST_KIND) == ST_UNKNOWN) {
        T diag, off;
        if (first) {
            level_stencil<T, false>(L, st, e, x, y, z, s, diag, off);
        } else {
            level_stencil<T>(L, st, e, x, y, z, s, diag, off);
        }
        T gs = ((T)L.h2 * rhs[c] + off) / diag;
        e[c] = first ? omega * gs : ((T)1 - omega) * e[c] + omega * gs;
    }
}

// Residual of level l at its unknown cells, restricted to level l+1 as the
// mean of the 8 children (children that are not unknowns contribute 0).
template <class T>
__global__ void __launch_bounds__(128) k_residual_restrict(LevelDesc L, const uint8_t* st, const T* rhs,
                                                           const T* e, int cnx, int cny, int cnz,
                                                           const uint8_t* cst, T* crhs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y, k = blockIdx.z;
    if (i >= cnx) return;
    T sum = (T)0;
    for (int dk = 0; dk < 2; dk++)
        for (int dj = 0; dj < 2; dj++)
            for (int di = 0; di < 2; di++) {
                int x = 2 * i + di, y = 2 * j + dj, z = 2 * k + dk;
                long long c = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
                uint8_t s = st[c];
                T r = (T)0;
                if ((s & ST_KIND) == ST_UNKNOWN) {
                    T diag, off;
                    level_stencil<T>(L, st, e, x, y, z, s, diag, off);
                    T Ae = (diag * e[c] - off) / (T)L.h2;
                    r = rhs[c] - Ae;
                }
                sum += r;
            }
    long long C = (long long)i + (long long)cnx * ((long long)j + (long long)cny * k);
    crhs[C] = ((cst[C] & ST_KIND) == ST_UNKNOWN) ? sum / (T)8 : (T)0;
    (void)cnz;
}

// e_l += e_{l+1}(parent) at unknown cells whose parent is an unknown
// (piecewise-constant prolongation).
template <class T>
__global__ void __launch_bounds__(128) k_prolong(LevelDesc L, const uint8_t* st, T* e, int cnx, int cny,
                                                 const uint8_t* cst, const T* ce) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    long long c = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
    long long C = (long long)(x >> 1) + (long long)cnx * ((long long)(y >> 1) + (long long)cny * (z >> 1));
    if ((st[c] & ST_KIND) == ST_UNKNOWN && (cst[C] & ST_KIND) == ST_UNKNOWN) e[c] += ce[C];
}

// Coarsest level: one thread block holds the level in shared memory and
// runs `sweeps` red-black sweeps from a zero iterate.
template <class T>
__global__ void __launch_bounds__(1024) k_coarse_solve(LevelDesc L, const uint8_t* st, const T* rhs, T* e,
                                                       int sweeps, T omega) {
    extern __shared__ unsigned char smem[];
    int n = L.nx * L.ny * L.nz;
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
                int x = i % L.nx, y = (i / L.nx) % L.ny, z = i / (L.nx * L.ny);
                if (((x + y + z) & 1) != colour) continue;
                uint8_t k = ss[i];
                if ((k & ST_KIND) != ST_UNKNOWN) continue;
                T diag, off;
                level_stencil<T>(L, ss, se, x, y, z, k, diag, off);
                T gs = ((T)L.h2 * sr[i] + off) / diag;
                se[i] = ((T)1 - omega) * se[i] + omega * gs;
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) e[i] = se[i];
}

template <class T>
__global__ void k_zero(T* p, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (T)0;
}

template <class T>
__global__ void k_correct(long long N, const uint8_t* st0, const T* e, double* psi) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    if ((st0[c] & ST_KIND) == ST_UNKNOWN) psi[c] += (double)e[c];
}

// --- EDL field and body force (Sec. 5.6) ---

// Value across face (a, side) of unknown cell c for a D3Q7 central
// difference: neighbour value, or the boundary value extrapolated from the
// cell (Dirichlet: 2 v - psi_c; Neumann: psi_c + sigma/eps; wall: psi_c).
__device__ __forceinline__ double face_value(const Grid& g, const Solver& s, const double* psi,
                                             const int32_t* owner, const DParticle* part, const int* kind,
                                             int x, int y, int z, double pc, int a, int side) {
    int d[3] = {0, 0, 0};
    d[a] = side;
    long long nb;
    if (!neighbour(g, x, y, z, d[0], d[1], d[2], nb)) {
        int face = 2 * a + (side > 0 ? 1 : 0);
        return s.pot_bc[face] == ES_POT_DIRICHLET ? 2.0 * s.pot_val[face] - pc : pc;
    }
    int o = owner[nb];
    if (o < 0) return psi[nb];
    if (kind[o] == ES_KIND_ZETA) return 2.0 * part[o].zeta - pc;
    return pc + part[o].sigma / s.eps;
}

template <class S>
__global__ void __launch_bounds__(128) k_body_force(Grid g, Solver s, double Ex, double Ey, double Ez,
                                                    const double* psi, const uint8_t* flags,
                                                    const int32_t* owner, const DParticle* part,
                                                    const int* kind, S* fb) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    long long c = lin(g, x, y, z);
    uint8_t fl = flags[c];
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;
    if (!(fl & F_SOLID)) {
        double pc = psi[c];
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        if (!(fl & F_NEAR19)) {
            // isotropic D3Q19 gradient (1/c_s^2) sum_q w_q psi(x + e_q) e_q
#pragma unroll
            for (int q = 1; q < 19; q++) {
                long long nb;
                neighbour(g, x, y, z, cx(q), cy(q), cz(q), nb);
                double v = wq(q) * psi[nb];
                g0 += v * cx(q);
                g1 += v * cy(q);
                g2 += v * cz(q);
            }
            g0 *= 3.0;
            g1 *= 3.0;
            g2 *= 3.0;
        } else {
            g0 = 0.5 * (face_value(g, s, psi, owner, part, kind, x, y, z, pc, 0, 1) -
                        face_value(g, s, psi, owner, part, kind, x, y, z, pc, 0, -1));
            g1 = 0.5 * (face_value(g, s, psi, owner, part, kind, x, y, z, pc, 1, 1) -
                        face_value(g, s, psi, owner, part, kind, x, y, z, pc, 1, -1));
            g2 = 0.5 * (face_value(g, s, psi, owner, part, kind, x, y, z, pc, 2, 1) -
                        face_value(g, s, psi, owner, part, kind, x, y, z, pc, 2, -1));
        }
        double rho_e = -s.kappa * s.kappa * s.eps * pc;  // Eq. ChrgDensDHA
        f0 = rho_e * (Ex - g0);
        f1 = rho_e * (Ey - g1);
        f2 = rho_e * (Ez - g2);
    }
    fb[c] = (S)f0;
    fb[g.N + c] = (S)f1;
    fb[2 * g.N + c] = (S)f2;
}

LevelDesc level_desc(const es_ctx* c, int l) {
    LevelDesc L;
    L.nx = c->ln[l][0];
    L.ny = c->ln[l][1];
    L.nz = c->ln[l][2];
    for (int a = 0; a < 3; a++) L.per[a] = c->g.per[a];
    for (int f = 0; f < 6; f++) L.pot_bc[f] = c->S.pot_bc[f];
    double h = (double)(1 << l);
    L.h2 = h * h;
    L.diag0 = 6.0 + c->S.kappa * c->S.kappa * h * h;
    return L;
}

size_t coarse_smem_bytes(const es_ctx* c, size_t tsize) {
    size_t n = (size_t)c->ln[c->L - 1][0] * c->ln[c->L - 1][1] * c->ln[c->L - 1][2];
    return n * (2 * tsize + 1);
}

template <class T>
cudaError_t vcycle_level(es_ctx* c, int l) {
    LevelDesc L = level_desc(c, l);
    T* e = (T*)c->e[l];
    T* rhs = (T*)c->rhs[l];
    const uint8_t* st = c->st[l];
    T omega = (T)c->P.omega;
    long long Nl = (long long)L.nx * L.ny * L.nz;
    dim3 blk(128);
    dim3 half(((L.nx + 1) / 2 + 127) / 128, L.ny, L.nz);
    dim3 full((L.nx + 127) / 128, L.ny, L.nz);
    if (l == c->L - 1) {
        size_t sm = coarse_smem_bytes(c, sizeof(T));
        if (sm <= 200 * 1024) {
            k_coarse_solve<T><<<1, 1024, sm, c->stream>>>(L, st, rhs, e, c->P.coarse_sweeps, omega);
            count(c);
        } else {
            count(c, 2 * c->P.coarse_sweeps + (c->P.coarse_sweeps == 0));
            if (c->P.coarse_sweeps == 0) k_zero<T><<<(unsigned)((Nl + 255) / 256), 256, 0, c->stream>>>(e, Nl);
            for (int s = 0; s < c->P.coarse_sweeps; s++) {
                k_smooth<T><<<half, blk, 0, c->stream>>>(L, st, rhs, e, 0, s == 0, omega);
                k_smooth<T><<<half, blk, 0, c->stream>>>(L, st, rhs, e, 1, 0, omega);
            }
        }
        return cudaGetLastError();
    }
    count(c, 2 * c->P.nu1 + 2 * c->P.nu2 + 2 + (c->P.nu1 == 0));
    if (c->P.nu1 == 0) k_zero<T><<<(unsigned)((Nl + 255) / 256), 256, 0, c->stream>>>(e, Nl);
    for (int s = 0; s < c->P.nu1; s++) {
        k_smooth<T><<<half, blk, 0, c->stream>>>(L, st, rhs, e, 0, s == 0, omega);
        k_smooth<T><<<half, blk, 0, c->stream>>>(L, st, rhs, e, 1, 0, omega);
    }
    const int* m = c->ln[l + 1];
    dim3 cgrid((m[0] + 127) / 128, m[1], m[2]);
    k_residual_restrict<T><<<cgrid, blk, 0, c->stream>>>(L, st, rhs, e, m[0], m[1], m[2], c->st[l + 1],
                                                         (T*)c->rhs[l + 1]);
    cudaError_t err = vcycle_level<T>(c, l + 1);
    if (err != cudaSuccess) return err;
    k_prolong<T><<<full, blk, 0, c->stream>>>(L, st, e, m[0], m[1], c->st[l + 1], (const T*)c->e[l + 1]);
    for (int s = 0; s < c->P.nu2; s++) {
        k_smooth<T><<<half, blk, 0, c->stream>>>(L, st, rhs, e, 0, 0, omega);
        k_smooth<T><<<half, blk, 0, c->stream>>>(L, st, rhs, e, 1, 0, omega);
    }
    return cudaGetLastError();
}

template <class T>
void set_coarse_smem(const es_ctx* c) {
    size_t sm = coarse_smem_bytes(c, sizeof(T));
    if (sm > 48 * 1024 && sm <= 200 * 1024)
        cudaFuncSetAttribute(k_coarse_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

}  // namespace

cudaError_t launch_outer_residual(es_ctx* c) {
    if (mixed(c))
        k_outer_residual<float><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            c->g, c->S, c->psi, c->st[0], c->owner, c->part, c->kind, (float*)c->rhs[0], c->partial);
    else
        k_outer_residual<double><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
            c->g, c->S, c->psi, c->st[0], c->owner, c->part, c->kind, (double*)c->rhs[0], c->partial);
    k_finalize_norm<<<1, 1024, 0, c->stream>>>(c->partial, c->red_blocks, c->d_norm);
    count(c, 2);
    return cudaGetLastError();
}

cudaError_t launch_vcycle(es_ctx* c) {
    if (mixed(c)) {
        set_coarse_smem<float>(c);
        return vcycle_level<float>(c, 0);
    }
    set_coarse_smem<double>(c);
    return vcycle_level<double>(c, 0);
}

cudaError_t launch_correct(es_ctx* c) {
    unsigned nb = (unsigned)((c->g.N + 255) / 256);
    if (mixed(c))
        k_correct<float><<<nb, 256, 0, c->stream>>>(c->g.N, c->st[0], (const float*)c->e[0], c->psi);
    else
        k_correct<double><<<nb, 256, 0, c->stream>>>(c->g.N, c->st[0], (const double*)c->e[0], c->psi);
    count(c);
    return cudaGetLastError();
}

cudaError_t launch_body_force(es_ctx* c) {
    const Grid& g = c->g;
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny, g.nz);
    const double* E = c->P.E_ext;
    if (mixed(c))
        k_body_force<float><<<grd, blk, 0, c->stream>>>(g, c->S, E[0], E[1], E[2], c->psi, c->flags, c->owner,
                                                        c->part, c->kind, (float*)c->fb);
    else
        k_body_force<double><<<grd, blk, 0, c->stream>>>(g, c->S, E[0], E[1], E[2], c->psi, c->flags, c->owner,
                                                         c->part, c->kind, (double*)c->fb);
    count(c);
    return cudaGetLastError();
}

}  // namespace es
