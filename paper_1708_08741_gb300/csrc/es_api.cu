// es_api.cu -- the C ABI of libes (declared in include/es.h): parameter
// validation, device state, and the host side of Algorithm 1 (Sec. 5.7).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "es_device.cuh"

using namespace es;

namespace {

thread_local std::string g_create_error;

int fail(es_ctx* c, int code, const std::string& msg) {
    if (c)
        c->err = msg;
    else
        g_create_error = msg;
    return code;
}

int cuda_fail(es_ctx* c, cudaError_t e, const char* where) {
    return fail(c, ES_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ES_CUDA(ctx, call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

// Parameter checks (the role of PhysicalCheck, Sec. 5.1).
int validate(const es_params* P, const es_particle* parts, int n, std::string& why) {
    if (!P) return why = "params is NULL", ES_EINVAL;
    if (n < 0 || (n > 0 && !parts)) return why = "bad particle array", ES_EINVAL;
    if (P->precision != ES_FP64 && P->precision != ES_MIXED32 && P->precision != ES_MIXED16)
        return why = "unknown precision", ES_EINVAL;
    if (P->levels < 1 || P->levels > ES_MAXLEV) return why = "levels must be in 1..12", ES_EINVAL;
    if (!(P->tau > 0.5)) return why = "tau must exceed 1/2", ES_EINVAL;
    if (!(P->eps > 0.0) || !(P->kappa >= 0.0)) return why = "eps must be > 0 and kappa >= 0", ES_EINVAL;
    if (P->smoother != ES_SMOOTH_FUSED && P->smoother != ES_SMOOTH_TWO_PASS) {
        why = "smoother must be ES_SMOOTH_FUSED or ES_SMOOTH_TWO_PASS";
        return ES_EINVAL;
    }
    if (P->mg_storage != ES_MG_NATIVE && P->mg_storage != ES_MG_FP16)
        return why = "mg_storage must be ES_MG_NATIVE or ES_MG_FP16", ES_EINVAL;
    if (P->mg_storage == ES_MG_FP16) {
        if (P->precision == ES_FP64) return why = "ES_MG_FP16 needs a reduced precision", ES_EINVAL;
        if (P->smoother != ES_SMOOTH_TWO_PASS) return why = "ES_MG_FP16 needs the two-pass smoother", ES_EINVAL;
        if (P->dims[0] % 4 != 0) return why = "ES_MG_FP16 needs dims[0] % 4 == 0", ES_EINVAL;
        if (P->levels < 2) return why = "ES_MG_FP16 needs levels >= 2", ES_EINVAL;
    }
    if (P->nu1 < 0 || P->nu2 < 0 || P->coarse_sweeps < 0 || P->max_cycles < 0)
        return why = "negative sweep or cycle count", ES_EINVAL;
    if (!(P->omega > 0.0 && P->omega < 2.0)) return why = "omega must be in (0, 2)", ES_EINVAL;
    if (!(P->rho_p_ratio > 0.0)) return why = "rho_p_ratio must be > 0", ES_EINVAL;
    for (int a = 0; a < 3; a++) {
        int d = P->dims[a];
        if (d < 1 || d > (1 << 20)) return why = "dims out of range", ES_EINVAL;
        if (d % (1 << (P->levels - 1)) != 0) return why = "dims must be multiples of 2^(levels-1)", ES_EINVAL;
        if (P->periodic[a] && d > 1 && ((d >> (P->levels - 1)) % 2) != 0)
            return why = "periodic extents must stay even on every level (red-black ordering)", ES_EINVAL;
    }
    if ((long long)P->dims[0] * P->dims[1] * P->dims[2] >= (1LL << 31))
        return why = "more than 2^31 - 1 cells (32-bit cell indices)", ES_EINVAL;
    for (int f = 0; f < 6; f++)
        if (P->pot_bc[f] != ES_POT_ZERO_FLUX && P->pot_bc[f] != ES_POT_DIRICHLET)
            return why = "unknown potential boundary kind", ES_EINVAL;
    for (int f = 0; f < 6; f++)
        if (P->wall_slip[f] != 0 && P->wall_slip[f] != 1) return why = "wall_slip entries must be 0 or 1", ES_EINVAL;
    if (!(P->phi_t >= 0.0) || std::isinf(P->phi_t)) return why = "phi_t must be finite and >= 0", ES_EINVAL;
    if (P->fine_layout != ES_LAYOUT_AUTO && P->fine_layout != ES_LAYOUT_NATURAL)
        return why = "fine_layout must be ES_LAYOUT_AUTO or ES_LAYOUT_NATURAL", ES_EINVAL;
    if (P->sweep_staging != ES_STAGE_REGISTERS && P->sweep_staging != ES_STAGE_BULK)
        return why = "sweep_staging must be ES_STAGE_REGISTERS or ES_STAGE_BULK", ES_EINVAL;
    if (P->lbm_block[0] != 0 || P->lbm_block[1] != 0) {
        const int bx = P->lbm_block[0], by = P->lbm_block[1];
        if (bx < 32 || bx > 256 || bx % 32 != 0 || by < 1 || bx * by > 256)
            return why = "lbm_block must be 0 x 0 or x in 32..256 (a multiple of 32) with x * y <= 256", ES_EINVAL;
    }
    if (P->near_list_cells < 0 || P->fast_update_cells < 0)
        return why = "near_list_cells and fast_update_cells must be >= 0", ES_EINVAL;
    if (P->phi_t > 0.0 && (P->precision != ES_FP64 || P->levels != 1))
        return why = "the nonlinear Poisson-Boltzmann form (phi_t > 0) needs ES_FP64 and levels == 1", ES_EINVAL;
    for (int p = 0; p < n; p++) {
        if (!(parts[p].R > 0.0)) return why = "particle radius must be > 0", ES_EINVAL;
        if (parts[p].kind != ES_KIND_ZETA && parts[p].kind != ES_KIND_CHARGE)
            return why = "unknown particle kind", ES_EINVAL;
        for (int a = 0; a < 3; a++)
            if (P->periodic[a] && !(2.0 * parts[p].R + 2.0 < (double)P->dims[a]))
                return why = "sphere too large for a periodic axis", ES_EINVAL;
    }
    return ES_OK;
}

DParticle to_device(const es_params& P, const es_particle& s, double sigma) {
    DParticle d;
    for (int a = 0; a < 3; a++) {
        d.x[a] = s.x[a];
        d.v[a] = s.v[a];
        d.w[a] = s.w[a];
    }
    d.R = s.R;
    d.zeta = s.zeta;
    d.q = s.q;
    d.sigma = sigma;
    // charge for F_C: q itself, or 4 pi R^2 sigma_s with the Debye-Hueckel
    // zeta-sigma relation (Eq. SurfChrgZetaRelationDebHuck)
    if (s.kind == ES_KIND_CHARGE) {
        d.qeff = s.q;
    } else {
        double sig = s.zeta * P.eps * (1.0 + P.kappa * s.R) / s.R;
        d.qeff = 4.0 * M_PI * s.R * s.R * sig;
    }
    d.mass = P.rho_p_ratio * 1.0 * (4.0 / 3.0) * M_PI * s.R * s.R * s.R;
    d.inertia = 0.4 * d.mass * s.R * s.R;
    return d;
}

// Stream stride of the PDF fields: N rounded up to 32 elements plus 1120
// elements (35 x 128 bytes in FP32), so that the same cell of the 19 streams
// does not sit at one power-of-two offset apart (DRAM partition camping).
long long pdf_stride(long long N) { return ((N + 31) / 32) * 32 + 1120; }

// The finest level's e and rhs are stored colour-split (see es.h, fine_layout).
bool colour_split(const es_params* P) {
    return P->precision != ES_FP64 && P->dims[0] % 8 == 0 && P->smoother == ES_SMOOTH_TWO_PASS &&
           P->mg_storage == ES_MG_NATIVE && P->levels >= 2 && P->fine_layout == ES_LAYOUT_AUTO;
}

// Level 1 colour-split as well: it is then not the coarsest level and its
// x extent keeps whole 8-cell spans.
bool colour_split1(const es_params* P) {
    return colour_split(P) && P->levels >= 3 && (P->dims[0] / 2) % 8 == 0;
}

size_t field_bytes(const es_params* P, int n, size_t* per_level) {
    long long N = (long long)P->dims[0] * P->dims[1] * P->dims[2];
    const size_t s = P->precision == ES_FP64 ? 8 : 4;  // arithmetic type
    size_t b = 0;
    b += 2 * 19 * pdf_stride(N) * pdf_bytes(P->precision);  // pdf ping-pong
    b += 3 * N * s;       // body force
    b += N * 8;           // psi: FP64, or float-float high and low parts
    b += N * 4 + N;       // owner, flags
    b += N * 4;           // list of fluid cells next to obstacles (body force)
    if (colour_split(P))  // per-colour update masks of the finest level
        b += (size_t)2 * P->dims[1] * P->dims[2] * ((P->dims[0] + 63) / 64) * 4;
    if (colour_split1(P))  // and of level 1
        b += (size_t)2 * (P->dims[1] / 2) * (P->dims[2] / 2) * ((P->dims[0] / 2 + 63) / 64) * 4;
    size_t lv = 0;
    for (int l = 0; l < P->levels; l++) {
        long long Nl = (long long)(P->dims[0] >> l) * (P->dims[1] >> l) * (P->dims[2] >> l);
        lv += Nl * (1 + 3 * s + 4);  // states, e, e2, rhs, near-cell lists (+ one row per segment)
        if (l == 0 && P->mg_storage == ES_MG_FP16) lv -= Nl * (s - 2);  // e as FP16
    }
    if (P->phi_t > 0.0) b += N * 8;  // linearised diagonal of the Poisson-Boltzmann stencil
    if (per_level) *per_level = lv;
    b += lv;
    b += (size_t)(n > 0 ? n : 1) * (sizeof(DParticle) + 9 * 8 + 4 + 4 + 6 * 8 + 14 * 4 + 12 * 8);
    b += res_partial_slots(P->dims[0], P->dims[1], 0) * 8 + 64;
    b += (size_t)kFlipCap * 4 + 3 * 256;  // flipped-cell list, its count, the moved flag
    if (colour_split(P)) b += (size_t)4 * kLocalCells * 4 + 1024;  // the local correction's scratch
    return b;
}

void* dev_alloc(es_ctx* c, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, c->user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        c->allocs.push_back(p);
        c->bytes += bytes;
    }
    return p;
}

void release(es_ctx* c) {
    cudaStreamSynchronize(c->stream);
    for (void* p : c->allocs) {
        if (c->alloc)
            c->freefn(p, c->user);
        else
            cudaFree(p);
    }
    c->allocs.clear();
    if (c->h_norm) cudaFreeHost(c->h_norm);
    if (c->h_status) cudaFreeHost(c->h_status);
    c->h_norm = nullptr;
    c->h_status = nullptr;
    for (void* h : {(void*)c->h_pset, (void*)c->h_pget, (void*)c->h_force})
        if (h) cudaFreeHost(h);
    c->h_pset = nullptr;
    c->h_pget = nullptr;
    c->h_force = nullptr;
    if (c->ev_stage) {
        cudaEventDestroy(c->ev_stage);
        c->ev_stage = nullptr;
    }
    for (auto& r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t ev : c->prof_pool) cudaEventDestroy(ev);
    c->prof_recs.clear();
    c->prof_pool.clear();
    for (int w = 0; w < 2; w++)
        if (c->vgraph[w]) {
            cudaGraphExecDestroy(c->vgraph[w]);
            c->vgraph[w] = nullptr;
        }
    if (c->ev_sync) {
        cudaEventDestroy(c->ev_sync);
        c->ev_sync = nullptr;
    }
}

// Reads the residual norm and the device status word (synchronises).
int read_norm_status(es_ctx* c, double* norm, int* status) {
    ES_CUDA(c, cudaMemcpyAsync(c->h_norm, c->d_norm, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    ES_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    *norm = c->h_norm[0];
    *status = c->h_status[0];
    return ES_OK;
}

int status_error(es_ctx* c, int st) {
    if (st & DS_OVERLAP) return fail(c, ES_EOVERLAP, "two particles claim the same cell");
    if (st & DS_WALLCUT) return fail(c, ES_EOVERLAP, "a sphere cuts a non-periodic wall");
    if (st & DS_TIMEOUT) return fail(c, ES_ETIMEOUT, "a kernel's wait for its asynchronous copies ran out");
    return ES_OK;
}

}  // namespace

namespace es {

ProfScope::ProfScope(es_ctx* c, const char* name, int level, double bytes) : c_(c), rec_(-1) {
    if (!c->prof) return;
    int slot = -1;
    for (size_t i = 0; i < c->prof_slots.size(); i++)
        if (c->prof_slots[i].level == level && c->prof_slots[i].name == name) slot = (int)i;
    if (slot < 0) {
        c->prof_slots.push_back({name, level, 0, 0.0});
        slot = (int)c->prof_slots.size() - 1;
    }
    c->prof_slots[slot].launches++;
    c->prof_slots[slot].bytes += bytes;
    cudaEvent_t ev[2];
    for (int k = 0; k < 2; k++) {
        if (!c->prof_pool.empty()) {
            ev[k] = c->prof_pool.back();
            c->prof_pool.pop_back();
        } else if (cudaEventCreate(&ev[k]) != cudaSuccess) {
            cudaGetLastError();
            if (k == 1) c->prof_pool.push_back(ev[0]);
            return;
        }
    }
    cudaEventRecord(ev[0], c->stream);
    c->prof_recs.push_back({slot, ev[0], ev[1]});
    rec_ = (int)c->prof_recs.size() - 1;
}

ProfScope::~ProfScope() {
    if (rec_ >= 0) cudaEventRecord(c_->prof_recs[rec_].b, c_->stream);
}

int field_components(int which) {
    if (which == ES_FIELD_PDF || which == ES_FIELD_PDF_LAST) return 19;
    if (which == ES_FIELD_U || which == ES_FIELD_FB) return 3;
    return 1;
}

int check_gather_args(es_ctx* c, int which, const int64_t* idx, int n, int max_n, const double* out) {
    if (!c || !idx || !out) return fail(c, ES_EINVAL, "NULL argument");
    if (n < 1 || n > max_n) return fail(c, ES_EINVAL, "n must be in 1.." + std::to_string(max_n));
    if (which < ES_FIELD_PSI || which > ES_FIELD_PDF_LAST) return fail(c, ES_EINVAL, "unknown field");
    if (which == ES_FIELD_PDF_LAST && c->last_src < 0) return fail(c, ES_EINVAL, "no LBM step yet");
    for (int i = 0; i < n; i++)
        if (idx[i] < 0 || idx[i] >= c->g.N) return fail(c, ES_EINVAL, "cell index out of range");
    return ES_OK;
}

}  // namespace es

extern "C" {

int es_create_with_allocator(const es_params* params, const es_particle* parts, int n, void* stream,
                             es_alloc_fn alloc, es_free_fn free_fn, void* user, es_ctx** out) {
    if (!out) return fail(nullptr, ES_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    int v = validate(params, parts, n, why);
    if (v != ES_OK) return fail(nullptr, v, why);
    if (alloc && !free_fn) return fail(nullptr, ES_EINVAL, "alloc given without free");
    es_ctx* c = new (std::nothrow) es_ctx();
    if (!c) return fail(nullptr, ES_ENOMEM, "host allocation failed");
    c->P = *params;
    c->stream = (cudaStream_t)stream;
    c->alloc = alloc;
    c->freefn = free_fn;
    c->user = user;
    c->np = n;
    c->g.nx = params->dims[0];
    c->g.ny = params->dims[1];
    c->g.nz = params->dims[2];
    for (int a = 0; a < 3; a++) c->g.per[a] = params->periodic[a] ? 1 : 0;
    c->rb0 = colour_split(params);
    c->rb1 = colour_split1(params);
    c->fb_lazy = false;
    c->bulk_smem_set = false;
    c->bulk_blocks = 0;
    c->slip = 0;
    for (int f = 0; f < 6; f++)
        if (!c->g.per[f / 2] && params->wall_slip[f]) c->slip |= 1 << f;
    c->g.N = (long long)c->g.nx * c->g.ny * c->g.nz;
    c->g.ps = pdf_stride(c->g.N);
    for (int f = 0; f < 6; f++) {
        c->S.pot_bc[f] = params->pot_bc[f];
        c->S.pot_val[f] = params->pot_val[f];
    }
    c->S.kappa = params->kappa;
    c->S.eps = params->eps;
    c->L = params->levels;
    for (int l = 0; l < c->L; l++)
        for (int a = 0; a < 3; a++) c->ln[l][a] = params->dims[a] >> l;
    // TRT rates (Sec. 4.1)
    c->lambda_e = -1.0 / params->tau;
    c->lambda_o = -8.0 * (2.0 - 1.0 / params->tau) / (8.0 - 1.0 / params->tau);
    c->cur = 0;
    c->last_src = -1;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
            cudaGetLastError();
            nsm = 152;
        }
        c->n_sm = nsm;
        c->device = dev;
    }
    c->red_blocks = 4 * c->n_sm;
    c->mg_rate = 0.15;
    c->e_scale = 1.0f;
    c->mapped_once = false;

    const long long N = c->g.N;
    const size_t s = mixed(c) ? 4 : 8;
    const int np1 = n > 0 ? n : 1;
    bool ok = true;
    auto A = [&](size_t bytes) {
        void* p = dev_alloc(c, bytes);
        if (!p) ok = false;
        return p;
    };
    c->pdf[0] = A(19 * c->g.ps * pdf_bytes(c->P.precision));
    c->pdf[1] = A(19 * c->g.ps * pdf_bytes(c->P.precision));
    c->fb = A(3 * N * s);
    c->psi = mixed(c) ? nullptr : (double*)A(N * 8);
    c->psi32 = mixed(c) ? (float*)A(N * 4) : nullptr;
    c->psi_lo = mixed(c) ? (float*)A(N * 4) : nullptr;
    c->dk = c->P.phi_t > 0.0 ? (double*)A(N * 8) : nullptr;
    c->owner = (int32_t*)A(N * 4);
    c->flags = (uint8_t*)A(N);
    for (int l = 0; l < c->L; l++) {
        long long Nl = (long long)c->ln[l][0] * c->ln[l][1] * c->ln[l][2];
        c->st[l] = (uint8_t*)A(Nl);
        c->e[l] = A(Nl * (l == 0 && c->P.mg_storage == ES_MG_FP16 ? 2 : s));
        c->e2[l] = A(Nl * s);
        {
            const long long rows = (long long)c->ln[l][1] * c->ln[l][2];
            // a segment holds one colour of rows = seg (mod kNearSegs)
            c->near_cap[l] = (int)(((rows + kNearSegs - 1) / kNearSegs) * ((c->ln[l][0] + 1) / 2));
            c->near_list[l] = (int*)A((size_t)2 * kNearSegs * c->near_cap[l] * 4);
        }
        c->rhs[l] = A(Nl * s);
    }
    c->part = (DParticle*)A(np1 * sizeof(DParticle));
    c->partf = mixed(c) ? (float*)A(np1 * 12 * sizeof(float)) : nullptr;
    c->pbc = mixed(c) ? (float*)A(np1 * 2 * sizeof(float)) : nullptr;
    c->mapped = (double*)A(np1 * 9 * 8);
    c->kind = (int*)A(np1 * 4);
    c->nfaces = (int*)A(np1 * 4);
    c->F = (double*)A(np1 * 3 * 8);
    c->T = (double*)A(np1 * 3 * 8);
    c->pstage = (double*)A(np1 * 12 * 8);
    c->partial = (double*)A(res_partial_slots(c->g.nx, c->g.ny, c->red_blocks) * 8);
    c->d_norm = (double*)A(64);
    c->near_count = (int*)A(2 * kNearSegs * ES_MAXLEV * 4);
    {
        const long long rows = (long long)c->g.ny * c->g.nz;
        c->bf_cap = (int)(((rows + kNearSegs - 1) / kNearSegs) * c->g.nx);
        c->bf_list = (int*)A((size_t)kNearSegs * c->bf_cap * 4);
        c->bf_count = (int*)A(kNearSegs * 4);
    }
    c->d_status = (int*)A(64);
    c->d_moved = (int*)A(64);
    c->flip_cap = kFlipCap;
    c->flip_list = (int*)A((size_t)kFlipCap * 4);
    c->flip_count = (int*)A(64);
    c->local_list = c->rb0 ? (int*)A((size_t)kLocalCells * 4) : nullptr;
    c->local_f = c->rb0 ? (float*)A((size_t)3 * kLocalCells * 4) : nullptr;
    c->local_meta = c->rb0 ? A(1024) : nullptr;
    c->res_valid = false;
    c->res_age = 0;
    c->rb_wpr = (c->g.nx + 63) / 64;
    c->rbmask = c->rb0 ? (uint32_t*)A((size_t)2 * c->g.ny * c->g.nz * c->rb_wpr * 4) : nullptr;
    c->rb_wpr1 = (c->ln[1][0] + 63) / 64;
    c->rbmask1 = c->rb1 ? (uint32_t*)A((size_t)2 * c->ln[1][1] * c->ln[1][2] * c->rb_wpr1 * 4) : nullptr;
    if (!ok) {
        release(c);
        delete c;
        return fail(nullptr, ES_ENOMEM, "device allocation failed");
    }
    if (cudaMallocHost(&c->h_norm, 64) != cudaSuccess || cudaMallocHost(&c->h_status, 64) != cudaSuccess ||
        cudaMallocHost(&c->h_pset, np1 * 12 * 8) != cudaSuccess ||
        cudaMallocHost(&c->h_pget, np1 * sizeof(DParticle)) != cudaSuccess ||
        cudaMallocHost(&c->h_force, np1 * 6 * 8) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_stage, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        release(c);
        delete c;
        return fail(nullptr, ES_ENOMEM, "pinned host allocation failed");
    }
    // initial state: fluid at rest, psi = 0, no obstacle cells
    cudaError_t e = cudaSuccess;
    std::vector<DParticle> hp(np1);
    std::vector<int> hk(np1, 0);
    std::vector<double> hm(9 * np1, 0.0);
    for (int p = 0; p < n; p++) {
        hp[p] = to_device(*params, parts[p], 0.0);
        hk[p] = parts[p].kind;
        c->h_R.push_back(parts[p].R);
        c->h_kind.push_back(parts[p].kind);
        for (int a = 0; a < 3; a++) {
            hm[9 * p + a] = parts[p].x[a];
            hm[9 * p + 3 + a] = parts[p].v[a];
            hm[9 * p + 6 + a] = parts[p].w[a];
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->part, hp.data(), np1 * sizeof(DParticle), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->kind, hk.data(), np1 * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->mapped, hm.data(), np1 * 9 * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->psi) e = cudaMemsetAsync(c->psi, 0, N * 8, c->stream);
    if (e == cudaSuccess && c->psi32) e = cudaMemsetAsync(c->psi32, 0, N * 4, c->stream);
    if (e == cudaSuccess && c->psi_lo) e = cudaMemsetAsync(c->psi_lo, 0, N * 4, c->stream);
    if (e == cudaSuccess && c->dk) e = cudaMemsetAsync(c->dk, 0, N * 8, c->stream);
    if (e == cudaSuccess && c->pbc) e = cudaMemsetAsync(c->pbc, 0, np1 * 2 * sizeof(float), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->fb, 0, 3 * N * s, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->F, 0, np1 * 3 * 8, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->T, 0, np1 * 3 * 8, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, 64, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_moved, 0, 64, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flip_count, 0, 64, c->stream);
    if (e == cudaSuccess) e = launch_init_flags(c);
    if (e == cudaSuccess) e = launch_coarse_states(c);
    if (e == cudaSuccess) e = launch_near_lists(c);
    if (e == cudaSuccess) e = launch_fill_rest(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        std::string msg = std::string("initialisation failed: ") + cudaGetErrorString(e);
        release(c);
        delete c;
        return fail(nullptr, ES_ECUDA, msg);
    }
    *out = c;
    return ES_OK;
}

int es_create(const es_params* params, const es_particle* parts, int n, void* stream, es_ctx** out) {
    return es_create_with_allocator(params, parts, n, stream, nullptr, nullptr, nullptr, out);
}

int es_destroy(es_ctx* c) {
    if (!c) return ES_OK;
    release(c);
    delete c;
    return ES_OK;
}

int es_map_particles(es_ctx* c) {
    if (!c) return fail(nullptr, ES_EINVAL, "ctx is NULL");
    ES_CUDA(c, launch_map(c));
    ES_CUDA(c, launch_coarse_states(c));
    ES_CUDA(c, launch_near_lists(c));
    return ES_OK;
}

// MIXED32/16: the FP32 V-cycles per correction are predicted to bring the
// residual to this fraction of the tolerance (a margin for the rate estimate).
constexpr double kCycleTarget = 0.85;
// The residual after a correction is updated in FP32 (r - A e) when the
// residual before it is within this factor of the tolerance.  The update
// forms A e from differences e_c - e_nb, so its rounding is ~1e-6 of the
// residual before the correction rather than of e (up to 1/kappa^2 larger);
// at 5000 x tol that stays near 0.5 % of the tolerance, inside the margin
// kCycleTarget leaves.
constexpr double kFastUpdate = 5000.0;
// A solve may start from the previous solve's residual patched around the
// spheres (k_flip_patch) this many times in a row; the next one forms
// it in full.  The residual carried between solves then holds at most this
// many corrections' FP32 updates, each ~1e-6 of a residual within
// kFastUpdate x tol, so its drift stays a small fraction of the tolerance.
constexpr int kResAgeMax = 8;
// (on small grids the float-float residual costs about a launch and the
// update's occasional second norm read costs a host round trip: the update
// is used from fast_update_cells cells on, default 2^21)
long long fast_update_cells(const es_ctx* c) {
    return c->P.fast_update_cells > 0 ? (long long)c->P.fast_update_cells : (long long)ES_FAST_UPDATE_CELLS;
}

int es_potential_solve(es_ctx* c, int forced_cycles, es_solve_info* info) {
    if (!c) return fail(nullptr, ES_EINVAL, "ctx is NULL");
    double norm;
    int st;
    // The residual of the previous solve's potential is still in the finest
    // right-hand side: form it again only around the spheres (unless one
    // moved far, which the device decides), and in full every kResAgeMax
    // solves, so that the FP32 updates of the corrections cannot drift.
    const bool patch = forced_cycles < 0 && c->rb0 && c->res_valid && c->res_age < kResAgeMax &&
                       c->g.N >= fast_update_cells(c);
    c->res_valid = false;
    ES_CUDA(c, launch_outer_residual(c, patch));
    c->res_age = patch ? c->res_age + 1 : 0;
    int rc = read_norm_status(c, &norm, &st);
    if (rc != ES_OK) return rc;
    if (st) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        return status_error(c, st);
    }
    const double norm0 = norm;
    if (!c->have_tol) {
        c->tol = c->P.res_rf * norm;
        c->have_tol = 1;
    }
    int cycles = 0;
    int result = ES_OK;
    for (;;) {
        if (std::isnan(norm) || std::isinf(norm)) {
            result = fail(c, ES_ENAN, "residual norm is not finite");
            break;
        }
        if (forced_cycles >= 0) {
            if (cycles >= forced_cycles) break;
        } else {
            // (an exactly zero residual is an exact solution; with a zero
            // first residual tol is zero and the test alone never ends)
            if (norm == 0.0 || !(norm >= c->tol)) break;
            if (cycles >= c->P.max_cycles) {
                result = fail(c, ES_ENOTCONVERGED, "max_cycles reached above tolerance");
                break;
            }
        }
        // V-cycles per correction: one in the FP64 form (the oracle's
        // iteration); in MIXED32 as many FP32 cycles, warm-started on the
        // same defect, as the running rate estimate says will bring the
        // residual below kCycleTarget x tolerance (at most 6, i.e. within
        // FP32 reach)
        int k = 1;
        if (mixed(c) && forced_cycles < 0) {
            double want = std::log(kCycleTarget * c->tol / norm) / std::log(c->mg_rate);
            k = (int)std::ceil(want);
            k = k < 1 ? 1 : (k > 6 ? 6 : k);
            if (k > c->P.max_cycles - cycles) k = c->P.max_cycles - cycles;
        }
        if (c->P.mg_storage == ES_MG_FP16) {
            // the FP16 correction holds s * e, s = sqrt(N) / ||r|| (the
            // residual's RMS scaled to one), fixed for this correction
            const double sc = norm > 0.0 ? std::sqrt((double)c->g.N) / norm : 1.0;
            c->e_scale = (float)(sc < 1e-30 ? 1e-30 : (sc > 1e30 ? 1e30 : sc));
        }
        for (int j = 0; j < k; j++) ES_CUDA(c, launch_vcycle(c, j > 0));
        const double before = norm;
        if (c->rb0 && forced_cycles < 0 && c->g.N >= fast_update_cells(c) && norm <= kFastUpdate * c->tol) {
            // near the tolerance: psi += e, then r -= A e (FP32 update, error
            // ~1e-6 of the residual before the correction); the float-float
            // residual is formed again only if the updated one is not yet
            // below the tolerance
            ES_CUDA(c, launch_residual_update(c, true));
            rc = read_norm_status(c, &norm, &st);
            if (rc != ES_OK) return rc;
            if (!(norm < c->tol) && !st) {
                ES_CUDA(c, launch_outer_residual(c));
                rc = read_norm_status(c, &norm, &st);
                if (rc != ES_OK) return rc;
            }
        } else {
            ES_CUDA(c, launch_correct(c));
            ES_CUDA(c, launch_outer_residual(c));
            rc = read_norm_status(c, &norm, &st);
            if (rc != ES_OK) return rc;
        }
        if (st) {
            cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
            return status_error(c, st);
        }
        cycles += k;
        if (norm > 0.0 && before > 0.0) {
            double observed = std::pow(norm / before, 1.0 / k);
            observed = observed < 0.01 ? 0.01 : (observed > 0.9 ? 0.9 : observed);
            c->mg_rate = std::exp(0.5 * std::log(c->mg_rate) + 0.5 * std::log(observed));
        }
    }
    if (info) {
        info->cycles = cycles;
        info->r_initial = norm0;
        info->r_final = norm;
        info->tol = c->tol;
    }
    // (every path of the loop leaves the residual of the final psi in the
    // finest right-hand side)
    c->res_valid = result == ES_OK;
    ES_CUDA(c, launch_body_force(c));
    return result;
}

int es_lbm_step(es_ctx* c) {
    if (!c) return fail(nullptr, ES_EINVAL, "ctx is NULL");
    ES_CUDA(c, launch_lbm(c));
    c->last_src = c->cur;
    c->cur = 1 - c->cur;
    return ES_OK;
}

int es_lbm_step_batch(es_ctx* const* ctxs, int n) {
    if (!ctxs || n < 1 || n > ES_LBM_BATCH_MAX) return fail(nullptr, ES_EINVAL, "need 1..ES_LBM_BATCH_MAX contexts");
    for (int i = 0; i < n; i++) {
        es_ctx* c = ctxs[i];
        if (!c) return fail(nullptr, ES_EINVAL, "a context is NULL");
        for (int j = 0; j < i; j++)
            if (ctxs[j] == c) return fail(c, ES_EINVAL, "a context appears twice in the batch");
        if (c->P.precision != ctxs[0]->P.precision) return fail(c, ES_EINVAL, "the contexts differ in precision");
        if (c->device != ctxs[0]->device) return fail(c, ES_EINVAL, "the contexts are on different devices");
        if (c->slip) return fail(c, ES_EINVAL, "free-slip walls are not batched");
    }
    const cudaError_t e = launch_lbm_batch(ctxs, n);
    if (e != cudaSuccess) return cuda_fail(ctxs[0], e, "es_lbm_step_batch");
    for (int i = 0; i < n; i++) {
        ctxs[i]->last_src = ctxs[i]->cur;
        ctxs[i]->cur = 1 - ctxs[i]->cur;
    }
    return ES_OK;
}

int es_forces(es_ctx* c, double* F, double* T, int on_device) {
    if (!c) return fail(nullptr, ES_EINVAL, "ctx is NULL");
    ES_CUDA(c, launch_forces(c));
    size_t b = (size_t)c->np * 3 * sizeof(double);
    if (c->np == 0) return ES_OK;
    if (on_device) {
        if (F) ES_CUDA(c, cudaMemcpyAsync(F, c->F, b, cudaMemcpyDeviceToDevice, c->stream));
        if (T) ES_CUDA(c, cudaMemcpyAsync(T, c->T, b, cudaMemcpyDeviceToDevice, c->stream));
        return ES_OK;
    }
    if (!F && !T) return ES_OK;
    // through the pinned staging buffer: F, then T
    double* h = c->h_force;
    if (F) ES_CUDA(c, cudaMemcpyAsync(h, c->F, b, cudaMemcpyDeviceToHost, c->stream));
    if (T) ES_CUDA(c, cudaMemcpyAsync(h + 3 * c->np, c->T, b, cudaMemcpyDeviceToHost, c->stream));
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    if (F) std::memcpy(F, h, b);
    if (T) std::memcpy(T, h + 3 * c->np, b);
    return ES_OK;
}

int es_advance(es_ctx* c) {
    if (!c) return fail(nullptr, ES_EINVAL, "ctx is NULL");
    ES_CUDA(c, launch_advance(c));
    return ES_OK;
}

int es_step(es_ctx* c, int forced_cycles, es_solve_info* info) {
    int rc = es_map_particles(c);
    if (rc != ES_OK) return rc;
    rc = es_potential_solve(c, forced_cycles, info);
    if (rc != ES_OK) return rc;
    rc = es_lbm_step(c);
    if (rc != ES_OK) return rc;
    rc = es_forces(c, nullptr, nullptr, 1);
    if (rc != ES_OK) return rc;
    return es_advance(c);
}

static size_t field_size(const es_ctx* c, int which) {
    long long N = c->g.N;
    switch (which) {
    case ES_FIELD_PSI:
    case ES_FIELD_RHO: return N * 8;
    case ES_FIELD_U:
    case ES_FIELD_FB: return 3 * N * 8;
    case ES_FIELD_PDF:
    case ES_FIELD_PDF_LAST: return 19 * N * 8;
    case ES_FIELD_OWNER: return N * 4;
    case ES_FIELD_FLAGS: return N;
    }
    return 0;
}

static double* io_buffer(es_ctx* c) {
    if (!c->io) c->io = dev_alloc(c, 19 * c->g.N * 8);
    return (double*)c->io;
}

int es_get_field(es_ctx* c, int which, void* dst, size_t bytes, int on_device) {
    if (!c || !dst) return fail(c, ES_EINVAL, "NULL argument");
    size_t need = field_size(c, which);
    if (need == 0 || bytes != need) return fail(c, ES_EINVAL, "unknown field or wrong size");
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const void* srcp = nullptr;
    if (which == ES_FIELD_PSI && !mixed(c)) srcp = c->psi;
    if (which == ES_FIELD_OWNER) srcp = c->owner;
    if (which == ES_FIELD_FLAGS) srcp = c->flags;
    if (!srcp) {
        double* buf = on_device ? (double*)dst : io_buffer(c);
        if (!buf) return fail(c, ES_ENOMEM, "staging buffer allocation failed");
        if (which == ES_FIELD_PDF) ES_CUDA(c, launch_get_pdf(c, c->cur, buf));
        if (which == ES_FIELD_PDF_LAST) {
            if (c->last_src < 0) return fail(c, ES_EINVAL, "no LBM step yet");
            ES_CUDA(c, launch_get_pdf(c, c->last_src, buf));
        }
        if (which == ES_FIELD_RHO) ES_CUDA(c, launch_get_moments(c, buf, nullptr));
        if (which == ES_FIELD_U) ES_CUDA(c, launch_get_moments(c, nullptr, buf));
        if (which == ES_FIELD_FB) ES_CUDA(c, launch_get_fb(c, buf));
        if (which == ES_FIELD_PSI) ES_CUDA(c, launch_join_psi(c, buf));
        srcp = on_device ? nullptr : buf;
    }
    if (srcp) ES_CUDA(c, cudaMemcpyAsync(dst, srcp, bytes, k, c->stream));
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    return ES_OK;
}

int es_gather(es_ctx* c, int which, const int64_t* idx, int n, double* out) {
    const int rc = check_gather_args(c, which, idx, n, 65536, out);
    if (rc != ES_OK) return rc;
    const size_t kmax = 65536;
    if (!c->gather) c->gather = dev_alloc(c, kmax * 8 + 19 * kmax * 8);
    if (!c->gather) return fail(c, ES_ENOMEM, "gather scratch allocation failed");
    long long* didx = (long long*)c->gather;
    double* dout = (double*)((char*)c->gather + kmax * 8);
    const int comps = field_components(which);
    ES_CUDA(c, cudaMemcpyAsync(didx, idx, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
    ES_CUDA(c, launch_gather(c, which, didx, n, dout));
    ES_CUDA(c, cudaMemcpyAsync(out, dout, (size_t)comps * n * 8, cudaMemcpyDeviceToHost, c->stream));
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    return ES_OK;
}

int es_set_field(es_ctx* c, int which, const void* src, size_t bytes, int on_device) {
    if (!c || !src) return fail(c, ES_EINVAL, "NULL argument");
    if (which != ES_FIELD_PSI && which != ES_FIELD_PDF && which != ES_FIELD_FB)
        return fail(c, ES_EINVAL, "field is read-only");
    if (bytes != field_size(c, which)) return fail(c, ES_EINVAL, "wrong size");
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (which == ES_FIELD_PSI) c->res_valid = false;  // (the carried residual belongs to the old psi)
    if (which == ES_FIELD_PSI && !mixed(c)) {
        ES_CUDA(c, cudaMemcpyAsync(c->psi, src, bytes, k, c->stream));
    } else {
        const double* dsrc = (const double*)src;
        if (!on_device) {
            double* buf = io_buffer(c);
            if (!buf) return fail(c, ES_ENOMEM, "staging buffer allocation failed");
            ES_CUDA(c, cudaMemcpyAsync(buf, src, bytes, cudaMemcpyHostToDevice, c->stream));
            dsrc = buf;
        }
        if (which == ES_FIELD_PDF) ES_CUDA(c, launch_set_pdf(c, dsrc));
        if (which == ES_FIELD_FB) ES_CUDA(c, launch_set_fb(c, dsrc));
        if (which == ES_FIELD_PSI) ES_CUDA(c, launch_split_psi(c, dsrc));
    }
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    return ES_OK;
}

int es_get_particles(es_ctx* c, es_particle* dst, int n) {
    if (!c || (n > 0 && !dst) || n != c->np) return fail(c, ES_EINVAL, "bad particle array");
    if (n == 0) return ES_OK;
    const DParticle* hp = c->h_pget;
    ES_CUDA(c, cudaMemcpyAsync(c->h_pget, c->part, n * sizeof(DParticle), cudaMemcpyDeviceToHost, c->stream));
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int p = 0; p < n; p++) {
        for (int a = 0; a < 3; a++) {
            dst[p].x[a] = hp[p].x[a];
            dst[p].v[a] = hp[p].v[a];
            dst[p].w[a] = hp[p].w[a];
        }
        dst[p].R = hp[p].R;
        dst[p].kind = c->h_kind[p];
        dst[p].zeta = hp[p].zeta;
        dst[p].q = hp[p].q;
    }
    return ES_OK;
}

int es_set_particles(es_ctx* c, const es_particle* src, int n) {
    if (!c || (n > 0 && !src) || n != c->np) return fail(c, ES_EINVAL, "bad particle array");
    std::string why;
    int v = validate(&c->P, src, n, why);
    if (v != ES_OK) return fail(c, v, why);
    if (n == 0) return ES_OK;
    // (the mapping updates flags and states near each sphere's surface only)
    for (int p = 0; p < n; p++)
        if (src[p].R != c->h_R[p] || src[p].kind != c->h_kind[p])
            return fail(c, ES_EINVAL, "a sphere's radius and kind are fixed after creation");
    // the staging buffer is reused once the previous call's copy out of it is done
    ES_CUDA(c, cudaEventSynchronize(c->ev_stage));
    double* h = c->h_pset;
    for (int p = 0; p < n; p++) {
        const DParticle d = to_device(c->P, src[p], 0.0);
        double* r = h + 12 * p;
        for (int a = 0; a < 3; a++) {
            r[a] = d.x[a];
            r[3 + a] = d.v[a];
            r[6 + a] = d.w[a];
        }
        r[9] = d.zeta;
        r[10] = d.q;
        r[11] = d.qeff;
    }
    ES_CUDA(c, cudaMemcpyAsync(c->pstage, h, (size_t)n * 12 * 8, cudaMemcpyHostToDevice, c->stream));
    ES_CUDA(c, cudaEventRecord(c->ev_stage, c->stream));
    // sigma is recomputed by the next mapping; the kernel keeps the current one meanwhile
    ES_CUDA(c, launch_set_particles(c));
    return ES_OK;
}

int es_set_forces(es_ctx* c, const double* F, const double* T, int n) {
    if (!c || n != c->np || (n > 0 && (!F || !T))) return fail(c, ES_EINVAL, "bad force arrays");
    if (n == 0) return ES_OK;
    ES_CUDA(c, cudaMemcpyAsync(c->F, F, n * 3 * 8, cudaMemcpyHostToDevice, c->stream));
    ES_CUDA(c, cudaMemcpyAsync(c->T, T, n * 3 * 8, cudaMemcpyHostToDevice, c->stream));
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    return ES_OK;
}

int es_synchronize(es_ctx* c) {
    if (!c) return fail(nullptr, ES_EINVAL, "ctx is NULL");
    ES_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    int st = c->h_status[0];
    if (st) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        return status_error(c, st);
    }
    return ES_OK;
}

int es_lattice(int* c57, double* w19) {
    if (!c57 || !w19) return ES_EINVAL;
    for (int q = 0; q < 19; q++) {
        c57[3 * q] = cx(q);
        c57[3 * q + 1] = cy(q);
        c57[3 * q + 2] = cz(q);
        w19[q] = wq(q);
    }
    return ES_OK;
}

uint64_t es_kernel_launches(const es_ctx* c) { return c ? (uint64_t)c->launches : 0; }

size_t es_device_bytes(const es_params* params, int n) {
    std::string why;
    if (!params || validate(params, nullptr, 0, why) != ES_OK) return 0;
    return field_bytes(params, n, nullptr);
}

int es_profile_start(es_ctx* c) {
    if (!c) return fail(nullptr, ES_EINVAL, "ctx is NULL");
    for (auto& r : c->prof_recs) {
        c->prof_pool.push_back(r.a);
        c->prof_pool.push_back(r.b);
    }
    c->prof_recs.clear();
    c->prof_slots.clear();
    c->prof = true;
    return ES_OK;
}

int es_profile_stop(es_ctx* c, es_kernel_time* out, int max, int* n) {
    if (!c) return fail(nullptr, ES_EINVAL, "ctx is NULL");
    if (!c->prof) return fail(c, ES_EINVAL, "profiling was not started");
    c->prof = false;
    ES_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<double> ms(c->prof_slots.size(), 0.0);
    for (auto& r : c->prof_recs) {
        float t = 0.0f;
        ES_CUDA(c, cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.slot] += t;
    }
    const int ns = (int)c->prof_slots.size();
    if (n) *n = ns;
    for (int i = 0; i < ns && i < max && out; i++) {
        std::memset(&out[i], 0, sizeof(es_kernel_time));
        std::strncpy(out[i].name, c->prof_slots[i].name.c_str(), sizeof(out[i].name) - 1);
        out[i].level = c->prof_slots[i].level;
        out[i].launches = c->prof_slots[i].launches;
        out[i].ms = ms[i];
        out[i].bytes = c->prof_slots[i].bytes;
    }
    return ES_OK;
}

const char* es_last_error(const es_ctx* c) {
    if (c) return c->err.c_str();
    return g_create_error.c_str();
}

}  // extern "C"
