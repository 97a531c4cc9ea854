// es_internal.cuh -- device data layout and kernel launchers of libes.
//
// Layout in HBM (N = nx*ny*nz cells, x fastest):
//   pdf[2]      19 streams of N populations (stride ps), ping-pong (pull
//               scheme).  FP64 form: f_q.  MIXED32 form: f_q - w_q as float,
//               which keeps FP32 resolution for the small deviations.
//   flags       N bytes: F_SOLID, F_NEAR19 (LBM / gradient fast path switch)
//   owner       N int32: sphere index of an obstacle cell, -1 fluid
//   psi         EDL potential, the outer iterate.  FP64 form: N doubles.
//               MIXED32 form: two float arrays psi32 (high part, also what
//               the FP32 kernels read) and psi_lo, a float-float value of
//               about 48 bits; the outer residual is formed in float-float
//               and rounded to the FP32 right-hand side rhs[0]
//   fb          3 x N body force in the storage type of the PDFs
//   st[l]       per multigrid level N_l bytes: kind (unknown / Dirichlet /
//               Neumann) and a "near boundary" bit; the stencil is implied by
//               these flags (quasi-constant stencil, Sec. 5.3)
//   e[l], rhs[l] per level N_l values of the inner multigrid type
//   particles   array of 128-byte records (DParticle) + kinds + forces
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/es.h"

#define ES_MAXLEV 12

namespace es {

// level-0 cell flags
enum : uint8_t { F_SOLID = 1, F_NEAR19 = 2 };
// multigrid level states: kind in the low two bits, near-boundary bit
enum : uint8_t { ST_UNKNOWN = 0, ST_DIR = 1, ST_NEU = 2, ST_KIND = 3, ST_NEAR = 4 };
// device status bits
enum : int { DS_OVERLAP = 1, DS_WALLCUT = 2, DS_TIMEOUT = 4 };

// D3Q19 (Sec. 4.1).  Direction q in 1..9 and q+9 are opposite.
__host__ __device__ constexpr int cx(int q) {
    constexpr int t[19] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, -1, 0, 0, -1, -1, -1, -1, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int cy(int q) {
    constexpr int t[19] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 0, -1, 0, -1, 1, 0, 0, -1, -1};
    return t[q];
}
__host__ __device__ constexpr int cz(int q) {
    constexpr int t[19] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 0, 0, -1, 1, -1, 1};
    return t[q];
}
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : (q <= 9 ? q + 9 : q - 9); }
__host__ __device__ constexpr double wq(int q) {
    return q == 0 ? 1.0 / 3.0 : ((q <= 3 || (q >= 10 && q <= 12)) ? 1.0 / 18.0 : 1.0 / 36.0);
}

// 128-byte particle record (FP64)
struct DParticle {
    double x[3], v[3], w[3];
    double R, zeta, q, sigma, qeff, mass, inertia;
};

// grid description passed by value to kernels
struct Grid {
    int nx, ny, nz;
    int per[3];
    long long N;
    long long ps;  // stride between PDF streams: N rounded up plus a pad that keeps
                   // the 19 streams off a common power-of-two alignment
};

struct Solver {
    int pot_bc[6];
    double pot_val[6];
    double kappa, eps;
};

}  // namespace es

struct es_ctx {
    es_params P;
    es::Grid g;
    es::Solver S;
    int np;
    cudaStream_t stream;
    es_alloc_fn alloc;
    es_free_fn freefn;
    void* user;
    std::vector<void*> allocs;
    // particles
    es::DParticle* part;   // current state
    float* partf;          // MIXED32: np x 12 floats (x, v, w) for the FP32 stream-collide
    double* mapped;        // np x 9: x, v, w used by the last mapping
    int* kind;
    int* nfaces;
    double *F, *T;         // np x 3
    double* pstage;        // np x 12: x, v, w, zeta, q, qeff of es_set_particles, copied in
    // fields
    void* pdf[2];
    int cur, last_src;
    uint8_t* flags;
    int32_t* owner;
    double* psi;     // FP64 form only
    float* psi32;    // MIXED32: high part of psi
    float* psi_lo;   // MIXED32: low part of psi
    double* dk;      // phi_t > 0: kappa^2 (cosh(psi / phi_t) - 1), the Newton diagonal shift
    float* pbc;      // MIXED32: np x 2, boundary value (2 zeta or sigma / eps) as float-float
    void* fb;
    // multigrid
    int L;
    int ln[ES_MAXLEV][3];
    uint8_t* st[ES_MAXLEV];
    void* e[ES_MAXLEV];
    void* rhs[ES_MAXLEV];
    void* e2[ES_MAXLEV];    // second iterate buffer: the fused sweep runs out of place
    int* near_list[ES_MAXLEV];  // near-boundary unknown cells per level: red segments, then black ones
    int near_cap[ES_MAXLEV];    // capacity of one segment
    int* near_count;            // device: 2 kNearSegs counts per level (red segments, then black)
    uint32_t* rbmask;           // colour-split finest level: per colour, one bit per cell (compact order,
                                // each row padded to rb_wpr words): 1 = interior unknown cell
    int rb_wpr;                 // mask words per row: ceil(nx / 64)
    uint32_t* rbmask1;          // the same for level 1 when it is colour-split as well (rb1)
    int rb_wpr1;
    int* bf_list;               // fluid cells with a non-fluid D3Q19 neighbour (level 0), kNearSegs segments
    int bf_cap;                 // capacity of one segment
    int* bf_count;              // device: kNearSegs counts
    int device;             // the CUDA device current at creation (the context's device)
    int n_sm;               // multiprocessors of the device
    int rb_blocks[2];       // resident fused-sweep blocks per SM (float, double); 0 = not queried
    double* partial;
    int red_blocks;
    double* d_norm;
    int* d_status;
    int* d_moved;    // device: 1 when a sphere moved half a cell or more since the last solve's start
                     // (or the flipped-cell list overflowed)
    int* flip_list;  // device: cells that changed between obstacle and fluid since then
    int* flip_count;
    int flip_cap;
    int* local_list;  // device scratch of the local correction at a solve's start (colour-split levels)
    float* local_f;   // 3 x kLocalCells floats
    void* local_meta; // the clusters of the flipped cells (LocalMeta, 1 KB)
    bool res_valid;  // the finest right-hand side holds the residual of the current psi (reduced forms)
    int res_age;     // solves started from a patched residual since the last full one
    double* h_norm;  // pinned: [0] norm
    int* h_status;   // pinned
    double* h_pset;  // pinned: np x 12, the staging of es_set_particles
    es::DParticle* h_pget;  // pinned: np records, es_get_particles
    double* h_force;        // pinned: np x 6, es_forces into host arrays
    cudaEvent_t ev_stage;   // the copy out of h_pset has completed
    double tol;
    int have_tol;
    double mg_rate;  // running estimate of the residual reduction per V-cycle
    float e_scale;   // ES_MG_FP16: scale of the finest level's stored correction
    int slip;        // bit f: face f (x-lo, x-hi, y-lo, ...) of a non-periodic axis is free-slip
    bool rb0;        // the finest level's e and rhs in the colour-split layout (reduced forms)
    bool rb1;        // level 1's as well (rb0, at least three levels, nx / 2 % 8 == 0)
    bool fb_lazy;    // f_b is derived from psi by the stream-collide (set by a solve when
                     // fb_fused); the stored field then holds it only after a read or
                     // at the cells next to obstacles
    bool mapped_once;  // the particles were mapped at least once (flags valid outside their shells)
    cudaGraphExec_t vgraph[2];          // the V-cycle from zero / warm-started, captured on first use
    unsigned long long vgraph_kernels[2];  // kernel launches in each graph
    bool vgraph_off;                    // capture failed once: launch directly
    cudaEvent_t ev_sync;                // orders the context's stream against a batched launch
    bool bulk_smem_set;                 // the staged half sweep's shared-memory size is set
    int bulk_blocks;                    // resident staged half-sweep blocks per SM; 0 = not queried
    std::vector<double> h_R;  // radii and kinds as created (fixed for the context's life)
    std::vector<int> h_kind;
    double lambda_e, lambda_o;
    size_t bytes;
    unsigned long long launches;  // kernels launched by this context
    void* io;        // lazily allocated staging buffer of 19 N doubles
    void* gather;    // lazily allocated gather scratch (indices + values)
    std::string err;
    // per-kernel event timing (es_profile_start / es_profile_stop)
    struct ProfSlot {
        std::string name;
        int level;
        int launches;
        double bytes;
    };
    struct ProfRec {
        int slot;
        cudaEvent_t a, b;
    };
    bool prof = false;
    std::vector<ProfSlot> prof_slots;
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;  // events of earlier sessions, reused
};

namespace es {

// ---- launchers (stream-ordered; return cudaGetLastError) ----
// mapping (es_map.cu)
cudaError_t launch_init_flags(es_ctx* c);
cudaError_t launch_map(es_ctx* c);
cudaError_t launch_coarse_states(es_ctx* c);
cudaError_t launch_near_lists(es_ctx* c);
// solver (es_solver.cu)
cudaError_t launch_outer_residual(es_ctx* c, bool patch = false);  // patch: see k_flip_patch
cudaError_t launch_vcycle(es_ctx* c, int warm);
cudaError_t launch_split_psi(es_ctx* c, const double* src);  // MIXED32: psi = src
cudaError_t launch_join_psi(es_ctx* c, double* dst);         // MIXED32: dst = psi
cudaError_t launch_correct(es_ctx* c);
cudaError_t launch_residual_update(es_ctx* c, bool correct);  // correct: psi += e in the same pass
cudaError_t launch_body_force(es_ctx* c);
cudaError_t launch_body_force_near(es_ctx* c);      // f_b at the listed cells next to obstacles
cudaError_t materialize_body_force(es_ctx* c);      // the whole stored f_b, when it is evaluated on the fly
bool fb_fused(const es_ctx* c);                     // the stream-collide evaluates f_b from psi
// lbm and particles (es_lbm.cu)
cudaError_t launch_lbm(es_ctx* c);
cudaError_t launch_lbm_batch(es_ctx* const* cs, int n);  // es_lbm_step_batch
cudaError_t launch_forces(es_ctx* c);
cudaError_t launch_advance(es_ctx* c);
cudaError_t launch_set_particles(es_ctx* c);  // part (and pbc) from pstage; sigma, mass, inertia kept
cudaError_t launch_fill_rest(es_ctx* c);
cudaError_t launch_get_pdf(es_ctx* c, int which_buf, double* dst);
cudaError_t launch_set_pdf(es_ctx* c, const double* src);
cudaError_t launch_get_moments(es_ctx* c, double* rho, double* u);
cudaError_t launch_set_fb(es_ctx* c, const double* src);
cudaError_t launch_get_fb(es_ctx* c, double* dst);
cudaError_t launch_gather(es_ctx* c, int which, const long long* idx, int n, double* out);

// Argument checks shared by es_gather and es_gather_noalloc (host only, no
// device work): ES_OK, or ES_EINVAL with the reason in c->err.
int check_gather_args(es_ctx* c, int which, const int64_t* idx, int n, int max_n, const double* out);
// Values per cell of a field (19 for the PDFs, 3 for U and FB, else 1).
int field_components(int which);

// The reduced-precision forms (FP32 arithmetic, float-float psi): MIXED32
// and MIXED16, which differ only in how the PDFs are stored.
inline bool mixed(const es_ctx* c) { return c->P.precision == ES_MIXED32 || c->P.precision == ES_MIXED16; }

// Bytes of one stored population.
inline size_t pdf_bytes(int precision) {
    return precision == ES_MIXED16 ? 2 : (precision == ES_MIXED32 ? 4 : 8);
}

// Near-cell lists are split by colour and by row (y + ny z) mod kNearSegs,
// each segment with its own counter, so that the list builder's atomics
// spread over that many addresses.
constexpr int kNearSegs = 64;
// blocks per 64 segments and per 64 SMs of a near-cell list pass (the
// passes are bound by the latency of their scattered loads: more threads in
// flight)
constexpr int kNearBlocks = 16;

// Blocks per segment (grid x) of a near-cell list pass: about 16 x 64 blocks
// per 64 SMs in all, whatever the segment count.
inline int near_grid_x(const es_ctx* c) {
    const int x = (c->n_sm + 63) / 64 * kNearBlocks * 64 / kNearSegs;
    return x < 1 ? 1 : x;
}

// Capacity of the per-block partial-sum array of the residual norm.
// Levels 0 and 1 may be stored colour-split (e and rhs: one colour's cells,
// then the other's, each in natural order; the states stay natural).
inline bool split_level(const es_ctx* c, int l) { return (l == 0 && c->rb0) || (l == 1 && c->rb1); }

constexpr int kFlipCap = 1 << 16;
// cells of the local correction's region and ring: at most 16 flipped cells, boxes of radius 9
constexpr int kLocalCells = 16 * 19 * 19 * 19;  // cells of the flipped-cell list (obstacle <-> fluid between solves)
constexpr int kResPartials = 8192;
// Partial-sum slots of the blocked residual norms: one per block of the
// marching residual passes (at most kResPartials planes of blocks, and a
// whole x-y plane of (32 lanes, 8 rows) blocks when that is more).
inline size_t res_partial_slots(int nx, int ny, int red_blocks) {
    const long long plane = (long long)((nx + 31) / 32) * ((ny + 7) / 8);
    long long n = plane > kResPartials ? plane : kResPartials;
    return (size_t)(n > red_blocks ? n : red_blocks);
}

// Brackets the launches made during its lifetime with CUDA events when the
// context is profiling (no-op otherwise); bytes: algorithmic bytes of the
// bracketed work.
class ProfScope {
   public:
    ProfScope(es_ctx* c, const char* name, int level, double bytes);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

   private:
    es_ctx* c_;
    int rec_;
};

// Every launch site adds its kernel count here.
inline void count(es_ctx* c, unsigned long long n = 1) { c->launches += n; }

}  // namespace es
