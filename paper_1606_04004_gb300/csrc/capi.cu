// C ABI of the library (declared in include/prunedq.h): object lifetime,
// argument checking, host <-> device marshalling.  The compute steps live in
// lattice.cu, apply_h.cu and krylov.cu.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "device_util.cuh"

namespace pq {

std::atomic<int64_t> g_launches{0};
static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}
void clear_error() { g_err.clear(); }

// caller's allocator (pq_set_allocator) and the number of live states
static pq_alloc_fn g_user_alloc = nullptr;
static pq_free_fn g_user_free = nullptr;
static void* g_user_ctx = nullptr;
static std::atomic<int64_t> g_live_states{0};

void* dev_alloc(size_t bytes, cudaStream_t st, bool async) {
    if (bytes == 0) bytes = 16;
    if (g_user_alloc) return g_user_alloc(bytes, (void*)st, g_user_ctx);
    void* p = nullptr;
    const cudaError_t e = async ? cudaMallocAsync(&p, bytes, st) : cudaMalloc(&p, bytes);
    return e == cudaSuccess ? p : nullptr;
}

void dev_free(void* p, cudaStream_t st, bool async) {
    if (!p) return;
    if (g_user_free) {
        g_user_free(p, (void*)st, g_user_ctx);
        return;
    }
    if (async) cudaFreeAsync(p, st);
    else cudaFree(p);
}

static void free_state(State* s) {
    if (!s) return;
    // a caller's allocator may hand the memory out again at once: let the
    // device finish with it first (cudaFree synchronises by itself)
    if (g_user_free) cudaDeviceSynchronize();
    if (s->rowinfo) dev_free(s->rowinfo, 0, false);
    if (s->h_na) cudaFreeHost(s->h_na);
    {
        void* pv[] = {s->pvbB64, s->pvbB32, s->pvbBh64, s->pvbBh32, s->pvbS64, s->pvbS32,
                      s->pvbSi64, s->pvbSi32, s->pvbT64, s->pvbT32, s->pvb_grid, s->pvb_vec,
                      s->fac_bra64};
        for (void* p : pv)
            dev_free(p, 0, false);
    }
    dev_free(s->vgrid64, 0, false);
    dev_free(s->vgrid32, 0, false);
    dev_free(s->gmat64, 0, false);
    dev_free(s->gmat32, 0, false);
    dev_free(s->gtmp, 0, false);
    void* ptrs[] = {s->keys,   s->psi,     s->psi_alt, s->bits,  s->bits_alt, s->off,
                    s->off_alt, s->rows,   s->planes,  s->leaders, s->cnt,    s->scan_tmp,
                    s->red_tmp, s->ks,     s->V,       s->T64,   s->T32,     s->pot64,
                    s->pot32,  s->fac64,   s->fac32,   s->io_in, s->io_out};
    for (void* p : ptrs)
        dev_free(p, 0, false);
    if (s->h_cnt) cudaFreeHost(s->h_cnt);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
    g_live_states.fetch_sub(1);
}

// Status of a CUDA call made while an object is being built (the caller
// frees what it built so far).
static pq_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PQ_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return PQ_ECUDA;
}

template <typename T>
static pq_status dalloc(T** p, size_t bytes) {
    *p = static_cast<T*>(dev_alloc(bytes, 0, false));
    if (!*p) {
        cudaGetLastError();   // clear a sticky allocation error
        set_error("device allocation of %zu bytes failed", bytes);
        return PQ_ENOMEM;
    }
    return PQ_OK;
}

// Device Hamiltonian tables from the basis' SoP.
static pq_status upload_hamiltonian(State& s) {
    const Basis& b = *s.basis;
    const int D = s.lat.D, lv = s.lead_virtual;
    const int nt = (int)b.pot_coef.size();
    std::vector<double> T((size_t)D * kMaxN * kMaxN, 0.0);
    for (int k = 0; k < b.D_user; ++k) {
        const int n = b.modes[k].n;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                T[(size_t)(k + lv) * kMaxN * kMaxN + i * kMaxN + j] =
                    b.kin_scale[k] * b.T[k][(size_t)i * n + j];
    }
    // Order the potential terms by which of the two last (tile) modes they
    // touch: neither, mode D-2 only, mode D-1 only, both.  The inner fibre pass
    // adds each group with the least work (see apply_h.cu).
    std::vector<int> order;
    for (int g = 0; g < 4; ++g) s.ngroup[g] = 0;
    for (int g = 0; g < 4; ++g)
        for (int t = 0; t < nt; ++t) {
            const uint32_t m = lv ? (b.pot_mask[t] << 1) : b.pot_mask[t];
            const int gt = ((m >> (D - 2)) & 1) + 2 * ((m >> (D - 1)) & 1);
            if (gt == g) {
                order.push_back(t);
                ++s.ngroup[g];
            }
        }
    // factor tables [term][mode][point] (identity factors hold 1), followed by
    // the term coefficients
    std::vector<double> P((size_t)std::max(nt, 1) * D * kMaxN + kMaxTerms, 0.0);
    for (int o = 0; o < nt; ++o) {
        P[(size_t)std::max(nt, 1) * D * kMaxN + o] = b.pot_coef[order[o]];
        const int t = order[o];
        for (int k = 0; k < D; ++k) {
            const int ku = k - lv;
            const int n = ku < 0 ? 1 : b.modes[ku].n;
            for (int i = 0; i < n; ++i) {
                P[((size_t)o * D + k) * kMaxN + i] =
                    ku < 0 ? 1.0 : b.pot_values[t][(size_t)ku * kMaxN + i];
            }
        }
    }
    std::vector<float> T32(T.begin(), T.end()), P32(P.begin(), P.end());
    pq_status rc;
    if ((rc = dalloc(&s.T64, T.size() * 8)) || (rc = dalloc(&s.T32, T.size() * 4)) ||
        (rc = dalloc(&s.pot64, P.size() * 8)) || (rc = dalloc(&s.pot32, P.size() * 4)))
        return rc;
    PQ_CUDA_TRY(cudaMemcpy(s.T64, T.data(), T.size() * 8, cudaMemcpyHostToDevice));
    PQ_CUDA_TRY(cudaMemcpy(s.T32, T32.data(), T32.size() * 4, cudaMemcpyHostToDevice));
    PQ_CUDA_TRY(cudaMemcpy(s.pot64, P.data(), P.size() * 8, cudaMemcpyHostToDevice));
    PQ_CUDA_TRY(cudaMemcpy(s.pot32, P32.data(), P32.size() * 4, cudaMemcpyHostToDevice));
    s.nterms = nt;
    return PQ_OK;
}

// Generic SoP (a basis with phase-space modes): every factor becomes a dense
// 1D matrix in the basis (congruence transform h^w = W^T h^chi W, Sec. 2.2
// Eq. pvb_H_trafo with B -> W for the orthogonal pW), single-factor terms are
// summed per mode, and terms with several factors keep their factor list for
// the pruned sequential transform (Sec. 2.2.2).
static pq_status upload_generic(State& s) {
    const Basis& b = *s.basis;
    const int D = s.lat.D, lv = s.lead_virtual;
    std::vector<std::vector<double>> mats;   // each kMaxN x kMaxN
    auto factor = [&](int ku, int kind, const std::vector<double>& vals) {
        const int n = b.modes[ku].n;
        std::vector<double> F((size_t)n * n, 0.0);
        if (kind == PQ_FACTOR_KINETIC) F = b.T[ku];
        else
            for (int i = 0; i < n; ++i) F[(size_t)i * n + i] = vals[i];
        if (!b.W[ku].empty()) {   // W^T F W
            const std::vector<double>& Wm = b.W[ku];
            std::vector<double> FW((size_t)n * n, 0.0), G((size_t)n * n, 0.0);
            for (int i = 0; i < n; ++i)
                for (int q = 0; q < n; ++q) {
                    double acc = 0.0;
                    for (int j = 0; j < n; ++j) acc += F[(size_t)i * n + j] * Wm[(size_t)j * n + q];
                    FW[(size_t)i * n + q] = acc;
                }
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q) {
                    double acc = 0.0;
                    for (int i = 0; i < n; ++i) acc += Wm[(size_t)i * n + p] * FW[(size_t)i * n + q];
                    G[(size_t)p * n + q] = acc;
                }
            F.swap(G);
        }
        std::vector<double> M((size_t)kMaxN * kMaxN, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) M[(size_t)i * kMaxN + j] = F[(size_t)i * n + j];
        return M;
    };
    for (int k = 0; k < kMaxD; ++k) s.gsingle[k] = -1;
    s.gplan.clear();
    for (const Basis::GTerm& t : b.gterms) {
        std::vector<int> fm;
        for (int ku = 0; ku < b.D_user; ++ku)
            if (t.kind[ku] != PQ_FACTOR_IDENTITY) fm.push_back(ku);
        if (fm.size() <= 1) {
            const int ku = fm.empty() ? b.D_user - 1 : fm[0];
            const int n = b.modes[ku].n;
            std::vector<double> M((size_t)kMaxN * kMaxN, 0.0);
            if (fm.empty())
                for (int i = 0; i < n; ++i) M[(size_t)i * kMaxN + i] = 1.0;
            else
                M = factor(ku, t.kind[ku], t.values[ku]);
            const int k = ku + lv;
            if (s.gsingle[k] < 0) {
                s.gsingle[k] = (int)mats.size();
                mats.push_back(std::vector<double>((size_t)kMaxN * kMaxN, 0.0));
            }
            std::vector<double>& acc = mats[s.gsingle[k]];
            for (size_t i = 0; i < acc.size(); ++i) acc[i] += t.coef * M[i];
            continue;
        }
        State::GPlan plan;
        plan.coef = t.coef;
        for (int f = (int)fm.size() - 1; f >= 0; --f) {   // last mode first
            plan.passes.push_back(State::GPass{fm[f] + lv, (int)mats.size()});
            mats.push_back(factor(fm[f], t.kind[fm[f]], t.values[fm[f]]));
        }
        s.gplan.push_back(plan);
    }
    const size_t nm = std::max<size_t>(mats.size(), 1);
    std::vector<double> M64(nm * kMaxN * kMaxN, 0.0);
    for (size_t m = 0; m < mats.size(); ++m)
        std::copy(mats[m].begin(), mats[m].end(), M64.begin() + m * kMaxN * kMaxN);
    std::vector<float> M32(M64.begin(), M64.end());
    pq_status rc;
    if ((rc = dalloc(&s.gmat64, M64.size() * 8)) || (rc = dalloc(&s.gmat32, M32.size() * 4)))
        return rc;
    PQ_CUDA_TRY(cudaMemcpy(s.gmat64, M64.data(), M64.size() * 8, cudaMemcpyHostToDevice));
    PQ_CUDA_TRY(cudaMemcpy(s.gmat32, M32.data(), M32.size() * 4, cudaMemcpyHostToDevice));
    if (!s.gplan.empty() && (rc = dalloc(&s.gtmp, 2 * s.cap * 16))) return rc;
    s.generic = true;
    (void)D;
    return PQ_OK;
}

// pvB matrices (Sec. 2.2): B, B^dagger, S = B^dagger B and the kinetic
// matrices as complex [D][kMaxN][kMaxN][2]; full-grid and work buffers.
static pq_status upload_pvb(State& s) {
    const Basis& b = *s.basis;
    const int D = s.lat.D, lv = s.lead_virtual;
    const size_t msz = (size_t)D * kMaxN * kMaxN * 2;
    std::vector<double> Bm(msz, 0.0), Bh(msz, 0.0), Sm(msz, 0.0), Tm(msz, 0.0), Si(msz, 0.0);
    double smax = 0.0;
    for (int k = 0; k < D; ++k) {
        const int ku = k - lv;
        const int n = ku < 0 ? 1 : b.modes[ku].n;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const size_t o = (((size_t)k * kMaxN + i) * kMaxN + j) * 2;
                if (ku < 0) {   // virtual size-1 mode: identity, no kinetic energy
                    Bm[o] = Bh[o] = Sm[o] = Si[o] = 1.0;
                    continue;
                }
                // S^-1 = (B^dagger B)^-1 = G^dagger G, since B = G^-dagger
                double sr = 0.0, si = 0.0;
                for (int q = 0; q < n; ++q) {
                    const size_t gi = ((size_t)q * n + i) * 2, gj = ((size_t)q * n + j) * 2;
                    const double ar = b.Gc[ku][gi], ai = -b.Gc[ku][gi + 1];
                    const double br = b.Gc[ku][gj], bi = b.Gc[ku][gj + 1];
                    sr += ar * br - ai * bi;
                    si += ar * bi + ai * br;
                }
                Si[o] = sr;
                Si[o + 1] = si;
                const size_t e = ((size_t)i * n + j) * 2, et = ((size_t)j * n + i) * 2;
                Bm[o] = b.Bc[ku][e];
                Bm[o + 1] = b.Bc[ku][e + 1];
                Bh[o] = b.Bc[ku][et];
                Bh[o + 1] = -b.Bc[ku][et + 1];
                Sm[o] = b.Sc[ku][e];
                Sm[o + 1] = b.Sc[ku][e + 1];
                smax = std::max(smax, std::hypot(Sm[o], Sm[o + 1]));
                Tm[o] = b.kin_scale[ku] * b.T[ku][(size_t)i * n + j];
            }
    }
    auto up = [&](const std::vector<double>& h, double** d64, float** d32) -> pq_status {
        std::vector<float> h32(h.begin(), h.end());
        pq_status rc;
        if ((rc = dalloc(d64, h.size() * 8)) || (rc = dalloc(d32, h.size() * 4))) return rc;
        PQ_CUDA_TRY(cudaMemcpy(*d64, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
        PQ_CUDA_TRY(cudaMemcpy(*d32, h32.data(), h32.size() * 4, cudaMemcpyHostToDevice));
        return PQ_OK;
    };
    pq_status rc;
    if ((rc = up(Bm, &s.pvbB64, &s.pvbB32)) || (rc = up(Bh, &s.pvbBh64, &s.pvbBh32)) ||
        (rc = up(Sm, &s.pvbS64, &s.pvbS32)) || (rc = up(Tm, &s.pvbT64, &s.pvbT32)) ||
        (rc = up(Si, &s.pvbSi64, &s.pvbSi32)))
        return rc;
    if ((rc = dalloc(&s.pvb_grid, (size_t)3 * s.lat.nfull * s.esize)) ||
        (rc = dalloc(&s.pvb_vec, (size_t)6 * s.cap * s.esize)))
        return rc;
    s.pvb_smax = smax > 0 ? smax : 1.0;
    s.pvb = true;
    return PQ_OK;
}

static pq_status create_state(const pq_basis* basis_, int precision, size_t capacity,
                              State** out) {
    const Basis* basis = reinterpret_cast<const Basis*>(basis_);
    if (!basis || !out) {
        set_error("null basis or output pointer");
        return PQ_EINVAL;
    }
    if (!basis->sop_set) {
        set_error("the basis has no Hamiltonian: call pq_set_sop first");
        return PQ_EINVAL;
    }
    if (precision != PQ_FP64 && precision != PQ_FP32MIX) {
        set_error("unknown precision %d", precision);
        return PQ_EINVAL;
    }
    State* s = new State();
    g_live_states.fetch_add(1);
    s->basis = basis;
    s->prec = precision;
    s->esize = precision == PQ_FP64 ? 16 : 8;
    s->lead_virtual = basis->D_user == 1 ? 1 : 0;
    Lattice& L = s->lat;
    L.D = basis->D_user + s->lead_virtual;
    for (int k = 0; k < L.D; ++k)
        L.n[k] = k < s->lead_virtual ? 1 : basis->modes[k - s->lead_virtual].n;
    pq_status rc = lattice_setup(*s);
    if (rc) {
        free_state(s);
        return rc;
    }
    // lattice axes of the neighbour rule: one per DVR mode, two (x, p) per
    // phase-space mode (function index a np + b: x slow, p fast)
    L.naxes = 0;
    for (int k = 0; k < L.D; ++k) {
        const int ku = k - s->lead_virtual;
        if (ku >= 0 && (!basis->W[ku].empty() || !basis->Bc[ku].empty())) {
            const int npl = basis->modes[ku].np_lattice;
            L.axis_n[L.naxes] = basis->modes[ku].nx_lattice;
            L.axis_stride[L.naxes++] = L.stride[k] * (uint32_t)npl;
            L.axis_n[L.naxes] = npl;
            L.axis_stride[L.naxes++] = L.stride[k];
        } else {
            L.axis_n[L.naxes] = L.n[k];
            L.axis_stride[L.naxes++] = L.stride[k];
        }
    }
    s->cap = capacity == 0 ? (size_t)L.nfull : std::min(capacity, (size_t)L.nfull);
    s->rows_cap = std::min(s->cap, (size_t)L.nrows);
    const size_t nw = L.nwords;
    if ((rc = dalloc(&s->keys, s->cap * 4)) || (rc = dalloc(&s->psi, s->cap * s->esize)) ||
        (rc = dalloc(&s->psi_alt, s->cap * s->esize)) || (rc = dalloc(&s->bits, nw * 8)) ||
        (rc = dalloc(&s->bits_alt, nw * 8)) || (rc = dalloc(&s->off, (nw + 1) * 4)) ||
        (rc = dalloc(&s->off_alt, (nw + 1) * 4)) || (rc = dalloc(&s->rows, s->rows_cap * 4)) ||
        (rc = dalloc(&s->planes, s->rows_cap * 4)) ||
        (rc = dalloc(&s->leaders, s->rows_cap * 4 * (size_t)std::max(1, L.D - 1))) ||
        (rc = dalloc(&s->cnt, CNT_SIZE * 8)) || (rc = dalloc(&s->scan_tmp, 1024 * 4)) ||
        (rc = dalloc(&s->red_tmp, (size_t)grid_size() * 8 * (2 * kMaxK + 8) * 8)) ||
        (rc = dalloc(&s->ks, sizeof(KrylovScalars)))) {
        free_state(s);
        return rc;
    }
    if (L.nlast <= 32 && L.nrows <= (1u << 28)) {
        if ((rc = dalloc(&s->rowinfo, (size_t)L.nrows * sizeof(uint2))) ||
            (rc = cuda_status(cudaMemset(s->rowinfo, 0, (size_t)L.nrows * sizeof(uint2)),
                              "clearing the row table"))) {
            free_state(s);
            return rc;
        }
    }
    if (cudaMallocHost((void**)&s->h_cnt, CNT_SIZE * 8) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        free_state(s);
        return PQ_ENOMEM;
    }
    if ((rc = cuda_status(cudaMemset(s->cnt, 0, CNT_SIZE * 8), "clearing the counters")) ||
        (rc = cuda_status(cudaMemset(s->bits, 0, nw * 8), "clearing the bitmap")) ||
        (rc = cuda_status(cudaMemset(s->off, 0, (nw + 1) * 4), "clearing the rank table")) ||
        (rc = cuda_status(cudaMemset(s->ks, 0, sizeof(KrylovScalars)), "clearing the scalars"))) {
        free_state(s);
        return rc;
    }
    if ((rc = basis->generic ? upload_generic(*s) : upload_hamiltonian(*s)) ||
        (basis->pvb && (rc = upload_pvb(*s)))) {
        free_state(s);
        return rc;
    }
    if (!basis->vgrid.empty()) {   // tabulated diagonal potential (DVR bases only)
        const size_t nv = basis->vgrid.size();
        std::vector<float> v32(basis->vgrid.begin(), basis->vgrid.end());
        if ((rc = dalloc(&s->vgrid64, nv * 8)) || (rc = dalloc(&s->vgrid32, nv * 4)) ||
            (rc = cuda_status(cudaMemcpy(s->vgrid64, basis->vgrid.data(), nv * 8,
                                         cudaMemcpyHostToDevice), "uploading the potential")) ||
            (rc = cuda_status(cudaMemcpy(s->vgrid32, v32.data(), nv * 4, cudaMemcpyHostToDevice),
                              "uploading the potential"))) {
            free_state(s);
            return rc;
        }
    }
    *out = s;
    return PQ_OK;
}

// An FP64 state on the basis, capacity and packet of s, with an empty active
// set: the adjoint sweep of a gradient whose forward run is FP32 (adjoint.cu).
pq_status make_fp64_twin(const State& s, State** out) {
    State* t = nullptr;
    pq_status rc = create_state(reinterpret_cast<const pq_basis*>(s.basis), PQ_FP64, s.cap, &t);
    if (rc) return rc;
    const size_t nf = (size_t)t->lat.D * kMaxN * 2;
    if ((rc = dalloc(&t->fac64, nf * 8)) || (rc = dalloc(&t->fac32, nf * 4)) ||
        (rc = cuda_status(cudaMemcpy(t->fac64, s.fac64, nf * 8, cudaMemcpyDeviceToDevice),
                          "copying the packet")) ||
        (rc = cuda_status(cudaMemcpy(t->fac32, s.fac32, nf * 4, cudaMemcpyDeviceToDevice),
                          "copying the packet"))) {
        free_state(t);
        return rc;
    }
    t->theta = s.theta;
    t->radius = s.radius;
    for (int k = 0; k < kMaxD; ++k) {
        t->q0[k] = s.q0[k];
        t->p0[k] = s.p0[k];
        t->width[k] = s.width[k];
    }
    *out = t;
    return PQ_OK;
}

void free_twin(State* t) { free_state(t); }

static pq_status check_capacity(State& s, cudaStream_t st) {
    PQ_CUDA_TRY(cudaMemcpyAsync(s.h_cnt, s.cnt, CNT_SIZE * 8, cudaMemcpyDeviceToHost, st));
    PQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (s.h_cnt[CNT_FAULT]) {
        set_error("bounds check failed: site %lld, index %lld, bound %lld",
                  (long long)s.h_cnt[CNT_FAULT], (long long)s.h_cnt[CNT_FAULT + 1],
                  (long long)s.h_cnt[CNT_FAULT + 2]);
        return PQ_EINVAL;
    }
    if (s.h_cnt[CNT_ERR] & 1) {
        set_error("active set of %lld points exceeds the capacity %zu",
                  (long long)s.h_cnt[CNT_NA], s.cap);
        return PQ_ECAPACITY;
    }
    return PQ_OK;
}

}  // namespace pq

using namespace pq;

#define PQ_API extern "C" __attribute__((visibility("default")))

PQ_API const char* pq_last_error(void) { return g_err.c_str(); }

PQ_API pq_status pq_set_allocator(pq_alloc_fn alloc, pq_free_fn free_fn, void* ctx) {
    clear_error();
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("give both an allocation and a release function, or neither");
        return PQ_EINVAL;
    }
    if (g_live_states.load() != 0) {
        set_error("the allocator cannot change while %lld state(s) exist",
                  (long long)g_live_states.load());
        return PQ_EINVAL;
    }
    g_user_alloc = alloc;
    g_user_free = free_fn;
    g_user_ctx = alloc ? ctx : nullptr;
    return PQ_OK;
}
PQ_API int64_t pq_launch_count(void) { return g_launches.load(); }

PQ_API pq_status pq_build_basis(const pq_mode_desc* modes, int D, pq_basis** out) {
    clear_error();
    if (!modes || !out) {
        set_error("null argument");
        return PQ_EINVAL;
    }
    if (D < 1 || D > kMaxD - 1) {
        set_error("D = %d outside 1..%d", D, kMaxD - 1);
        return PQ_EINVAL;
    }
    Basis* b = new Basis();
    b->D_user = D;
    b->modes.assign(modes, modes + D);
    b->x.resize(D);
    b->w.resize(D);
    b->T.resize(D);
    b->W.resize(D);
    b->Gc.resize(D);
    b->Bc.resize(D);
    b->Sc.resize(D);
    int npvb = 0;
    for (int k = 0; k < D; ++k) npvb += modes[k].kind == PQ_PVB;
    if (npvb != 0 && npvb != D) {
        set_error("a pvB basis must use pvB for every mode (mixed bases are not provided)");
        delete b;
        return PQ_ENOTSUP;
    }
    b->pvb = npvb == D;
    double full = 1;
    for (int k = 0; k < D; ++k) {
        pq_status rc = modes[k].kind == PQ_PW
                           ? build_pw_mode(modes[k], b->x[k], b->w[k], b->T[k], b->W[k])
                       : modes[k].kind == PQ_PVB
                           ? build_pvb_mode(modes[k], b->x[k], b->w[k], b->T[k], b->Gc[k], b->Bc[k],
                                            b->Sc[k])
                           : build_dvr_mode(modes[k], b->x[k], b->w[k], b->T[k]);
        if (modes[k].kind == PQ_PW) b->generic = true;
        if (rc) {
            delete b;
            return rc;
        }
        full *= modes[k].n;
    }
    if (full >= 4294967296.0) {
        set_error("lattice of %.0f points: the limit is 2^32", full);
        delete b;
        return PQ_EINVAL;
    }
    *out = reinterpret_cast<pq_basis*>(b);
    return PQ_OK;
}

PQ_API void pq_basis_free(pq_basis* basis) { delete reinterpret_cast<Basis*>(basis); }

PQ_API pq_status pq_basis_grid(const pq_basis* basis_, int mode, double* x, double* w) {
    clear_error();
    const Basis* b = reinterpret_cast<const Basis*>(basis_);
    if (!b || mode < 0 || mode >= b->D_user) {
        set_error("bad basis or mode");
        return PQ_EINVAL;
    }
    const int n = b->modes[mode].n;
    if (x) memcpy(x, b->x[mode].data(), n * sizeof(double));
    if (w) memcpy(w, b->w[mode].data(), n * sizeof(double));
    return PQ_OK;
}

PQ_API pq_status pq_basis_kinetic(const pq_basis* basis_, int mode, double* T) {
    clear_error();
    const Basis* b = reinterpret_cast<const Basis*>(basis_);
    if (!b || !T || mode < 0 || mode >= b->D_user) {
        set_error("bad basis, mode or output");
        return PQ_EINVAL;
    }
    const int n = b->modes[mode].n;
    memcpy(T, b->T[mode].data(), (size_t)n * n * sizeof(double));
    return PQ_OK;
}

PQ_API pq_status pq_basis_transform(const pq_basis* basis_, int mode, double* Wout) {
    clear_error();
    const Basis* b = reinterpret_cast<const Basis*>(basis_);
    if (!b || !Wout || mode < 0 || mode >= b->D_user) {
        set_error("bad basis, mode or output");
        return PQ_EINVAL;
    }
    const int n = b->modes[mode].n;
    if (b->W[mode].empty())
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) Wout[(size_t)i * n + j] = i == j ? 1.0 : 0.0;
    else
        memcpy(Wout, b->W[mode].data(), (size_t)n * n * sizeof(double));
    return PQ_OK;
}

PQ_API pq_status pq_set_potential_grid(pq_basis* basis_, const double* V, int64_t n) {
    clear_error();
    Basis* b = reinterpret_cast<Basis*>(basis_);
    if (!b) {
        set_error("null basis");
        return PQ_EINVAL;
    }
    if (b->generic || b->pvb) {
        set_error("a tabulated potential is provided for DVR bases only");
        return PQ_ENOTSUP;
    }
    if (!V) {
        b->vgrid.clear();
        return PQ_OK;
    }
    double full = 1;
    for (int k = 0; k < b->D_user; ++k) full *= b->modes[k].n;
    if ((double)n != full) {
        set_error("tabulated potential of %lld values for a lattice of %.0f points", (long long)n,
                  full);
        return PQ_EINVAL;
    }
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(V[i])) {
            set_error("tabulated potential value %lld is not finite", (long long)i);
            return PQ_EINVAL;
        }
    b->vgrid.assign(V, V + n);
    return PQ_OK;
}

PQ_API pq_status pq_set_sop(pq_basis* basis_, const pq_sop_term* terms, int nterms) {
    clear_error();
    Basis* b = reinterpret_cast<Basis*>(basis_);
    if (!b || (nterms > 0 && !terms) || nterms < 0) {
        set_error("bad basis or term list");
        return PQ_EINVAL;
    }
    const int D = b->D_user;
    if (b->generic) {
        std::vector<Basis::GTerm> gt;
        for (int t = 0; t < nterms; ++t) {
            const pq_sop_term& tm = terms[t];
            if (!tm.factors || !std::isfinite(tm.coef)) {
                set_error("term %d: no factors or non-finite coefficient", t);
                return PQ_EINVAL;
            }
            Basis::GTerm g;
            g.coef = tm.coef;
            g.kind.resize(D);
            g.values.resize(D);
            for (int k = 0; k < D; ++k) {
                const int kind = tm.factors[k].kind;
                if (kind != PQ_FACTOR_IDENTITY && kind != PQ_FACTOR_KINETIC && kind != PQ_FACTOR_DIAG) {
                    set_error("term %d mode %d: unknown factor kind %d", t, k, kind);
                    return PQ_EINVAL;
                }
                g.kind[k] = kind;
                if (kind == PQ_FACTOR_DIAG) {
                    if (!tm.factors[k].values) {
                        set_error("term %d mode %d: diagonal factor without values", t, k);
                        return PQ_EINVAL;
                    }
                    g.values[k].assign(tm.factors[k].values, tm.factors[k].values + b->modes[k].n);
                    for (double v : g.values[k])
                        if (!std::isfinite(v)) {
                            set_error("term %d mode %d: non-finite value", t, k);
                            return PQ_EINVAL;
                        }
                }
            }
            gt.push_back(g);
        }
        b->gterms = gt;
        b->sop_set = true;
        return PQ_OK;
    }
    std::vector<double> kin(D, 0.0), pc;
    std::vector<std::vector<double>> pv;
    std::vector<uint32_t> pm;
    for (int t = 0; t < nterms; ++t) {
        const pq_sop_term& tm = terms[t];
        if (!tm.factors) {
            set_error("term %d has no factors", t);
            return PQ_EINVAL;
        }
        int nkin = 0, kmode = -1, ndiag = 0;
        for (int k = 0; k < D; ++k) {
            const int kind = tm.factors[k].kind;
            if (kind == PQ_FACTOR_KINETIC) {
                ++nkin;
                kmode = k;
            } else if (kind == PQ_FACTOR_DIAG) {
                if (!tm.factors[k].values) {
                    set_error("term %d mode %d: diagonal factor without values", t, k);
                    return PQ_EINVAL;
                }
                ++ndiag;
            } else if (kind != PQ_FACTOR_IDENTITY) {
                set_error("term %d mode %d: unknown factor kind %d", t, k, kind);
                return PQ_EINVAL;
            }
        }
        if (!std::isfinite(tm.coef)) {
            set_error("term %d: non-finite coefficient", t);
            return PQ_EINVAL;
        }
        if (nkin > 1 || (nkin == 1 && ndiag > 0)) {
            set_error("term %d: a DVR term is either one kinetic factor or diagonal factors", t);
            return PQ_ENOTSUP;
        }
        if (nkin == 1) {
            kin[kmode] += tm.coef;
            continue;
        }
        std::vector<double> vals((size_t)D * kMaxN, 1.0);
        uint32_t mask = 0;
        for (int k = 0; k < D; ++k)
            if (tm.factors[k].kind == PQ_FACTOR_DIAG) mask |= 1u << k;
        for (int k = 0; k < D; ++k)
            if (tm.factors[k].kind == PQ_FACTOR_DIAG)
                for (int i = 0; i < b->modes[k].n; ++i) {
                    const double v = tm.factors[k].values[i];
                    if (!std::isfinite(v)) {
                        set_error("term %d mode %d: non-finite value", t, k);
                        return PQ_EINVAL;
                    }
                    vals[(size_t)k * kMaxN + i] = v;
                }
        pc.push_back(tm.coef);
        pv.push_back(vals);
        pm.push_back(mask);
    }
    if ((int)pc.size() > kMaxTerms) {
        set_error("%zu potential terms: at most %d", pc.size(), kMaxTerms);
        return PQ_ENOTSUP;
    }
    b->kin_scale = kin;
    b->pot_coef = pc;
    b->pot_values = pv;
    b->pot_mask = pm;
    b->sop_set = true;
    return PQ_OK;
}

PQ_API pq_status pq_init_packet(const pq_basis* basis_, const double* q0, const double* p0,
                                const double* width, double theta, int radius, int precision,
                                size_t capacity, pq_state** out) {
    clear_error();
    if (!q0 || !p0 || !width) {
        set_error("null packet parameter");
        return PQ_EINVAL;
    }
    if (!(theta >= 0) || !std::isfinite(theta)) {
        set_error("theta must be finite and >= 0");
        return PQ_EINVAL;
    }
    if (radius != PQ_RADIUS_1 && radius != PQ_RADIUS_SQRT2 && radius != PQ_RADIUS_2) {
        set_error("unknown neighbour rule %d (1: radius 1, 2: radius sqrt 2, 3: radius 2)", radius);
        return PQ_EINVAL;
    }
    const Basis* b = reinterpret_cast<const Basis*>(basis_);
    if (b)
        for (int k = 0; k < b->D_user; ++k)
            if (!(width[k] > 0)) {
                set_error("packet width of mode %d must be positive", k);
                return PQ_EINVAL;
            }
    State* s = nullptr;
    pq_status rc = create_state(basis_, precision, capacity, &s);
    if (rc) return rc;
    std::vector<double> fac;
    packet_factors(*b, q0, p0, width, fac, s->lead_virtual);
    std::vector<float> fac32(fac.begin(), fac.end());
    if ((rc = dalloc(&s->fac64, fac.size() * 8)) || (rc = dalloc(&s->fac32, fac32.size() * 4)) ||
        (rc = cuda_status(cudaMemcpy(s->fac64, fac.data(), fac.size() * 8, cudaMemcpyHostToDevice),
                          "uploading the packet")) ||
        (rc = cuda_status(cudaMemcpy(s->fac32, fac32.data(), fac32.size() * 4,
                                     cudaMemcpyHostToDevice), "uploading the packet"))) {
        free_state(s);
        return rc;
    }
    if (b->pvb) {   // bra of the autocorrelation: B^dagger f per mode
        std::vector<double> bra;
        Basis tmp = *b;
        tmp.Gc = b->Bc;
        packet_factors(tmp, q0, p0, width, bra, s->lead_virtual);
        if ((rc = dalloc(&s->fac_bra64, bra.size() * 8)) ||
            (rc = cuda_status(cudaMemcpy(s->fac_bra64, bra.data(), bra.size() * 8,
                                         cudaMemcpyHostToDevice), "uploading the packet bra"))) {
            free_state(s);
            return rc;
        }
    }
    s->theta = theta;
    s->radius = radius;
    for (int k = 0; k < b->D_user; ++k) {
        s->q0[k] = q0[k];
        s->p0[k] = p0[k];
        s->width[k] = width[k];
    }
    cudaStream_t st = 0;
    if ((rc = init_bits_from_packet(*s, theta, st)) || (rc = check_capacity(*s, st)) ||
        (rc = set_psi_from_packet(*s, st)) ||
        (rc = s->pvb ? pvb_observe_current(*s, theta, st) : observe_launch(*s, theta, st))) {
        free_state(s);
        return rc;
    }
    *out = reinterpret_cast<pq_state*>(s);
    return PQ_OK;
}

PQ_API void pq_state_free(pq_state* state) { free_state(reinterpret_cast<State*>(state)); }

PQ_API pq_status pq_state_load(pq_state* state, const int64_t* idx, int64_t n, const void* psi) {
    clear_error();
    State* s = reinterpret_cast<State*>(state);
    if (!s || n < 0 || (n > 0 && !idx)) {
        set_error("bad state or index list");
        return PQ_EINVAL;
    }
    if ((size_t)n > s->cap) {
        set_error("%lld points exceed the capacity %zu", (long long)n, s->cap);
        return PQ_ECAPACITY;
    }
    std::vector<uint32_t> k32((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        if (idx[i] < 0 || idx[i] >= (int64_t)s->lat.nfull || (i > 0 && idx[i] <= idx[i - 1])) {
            set_error("index %lld at position %lld is out of the lattice or not increasing",
                      (long long)idx[i], (long long)i);
            return PQ_EINVAL;
        }
        k32[i] = (uint32_t)idx[i];
    }
    uint32_t* dk = nullptr;
    pq_status rc = dalloc(&dk, (size_t)n * 4);
    if (rc) return rc;
    if (n > 0)   // an empty list has no host data to copy
        rc = cuda_status(cudaMemcpy(dk, k32.data(), (size_t)n * 4, cudaMemcpyHostToDevice),
                         "uploading the index list");
    if (!rc) rc = load_set(*s, dk, n, 0);
    cudaDeviceSynchronize();
    dev_free(dk, 0, false);
    if (rc) return rc;
    if (psi)
        PQ_CUDA_TRY(cudaMemcpy(s->psi, psi, (size_t)n * s->esize, cudaMemcpyHostToDevice));
    else
        PQ_CUDA_TRY(cudaMemset(s->psi, 0, (size_t)std::max<int64_t>(n, 1) * s->esize));
    return check_capacity(*s, 0);
}

PQ_API pq_status pq_state_size(const pq_state* state, int64_t* n_active) {
    clear_error();
    State* s = const_cast<State*>(reinterpret_cast<const State*>(state));
    if (!s || !n_active) {
        set_error("null argument");
        return PQ_EINVAL;
    }
    PQ_CUDA_TRY(cudaDeviceSynchronize());
    PQ_CUDA_TRY(cudaMemcpy(s->h_cnt, s->cnt, CNT_SIZE * 8, cudaMemcpyDeviceToHost));
    *n_active = std::min<int64_t>(s->h_cnt[CNT_NA], (int64_t)s->cap);
    return PQ_OK;
}

PQ_API pq_status pq_state_read(const pq_state* state, int64_t* idx, void* psi) {
    clear_error();
    const State* s = reinterpret_cast<const State*>(state);
    int64_t n = 0;
    pq_status rc = pq_state_size(state, &n);
    if (rc) return rc;
    if (idx && n > 0) {
        std::vector<uint32_t> k32((size_t)n);
        PQ_CUDA_TRY(cudaMemcpy(k32.data(), s->keys, (size_t)n * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) idx[i] = k32[i];
    }
    if (psi && n > 0)
        PQ_CUDA_TRY(cudaMemcpy(psi, s->psi, (size_t)n * s->esize, cudaMemcpyDeviceToHost));
    return PQ_OK;
}

PQ_API pq_status pq_state_psi_device(const pq_state* state, void** psi) {
    clear_error();
    const State* s = reinterpret_cast<const State*>(state);
    if (!s || !psi) {
        set_error("null argument");
        return PQ_EINVAL;
    }
    *psi = s->psi;
    return PQ_OK;
}

// <in, out> over the active set: per-block partials (Re, Im; FP64 sums of the
// per-element products), then one block adds them in block order.
constexpr int kVhvThreads = 256;
template <typename V>
__global__ void __launch_bounds__(kVhvThreads) k_vhv_partials(const V* __restrict__ x,
                                                              const V* __restrict__ y,
                                                              const int64_t* na, int64_t cap,
                                                              double* partials) {
    const int64_t n = min(*na, cap);
    double re = 0.0, im = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const V a = x[p], b = y[p];
        re += (double)a.x * b.x + (double)a.y * b.y;   // conj(a) b
        im += (double)a.x * b.y - (double)a.y * b.x;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    __shared__ double sh[2][kVhvThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = re;
        sh[1][threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < kVhvThreads / 32; ++w) t += sh[threadIdx.x][w];
        partials[2 * blockIdx.x + threadIdx.x] = t;
    }
}

__global__ void k_vhv_sum(const double* partials, int G, double* out) {
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int b = 0; b < G; ++b) t += partials[2 * b + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

PQ_API pq_status pq_apply_H(const pq_state* state, const void* in, void* out, int precision,
                            double* out_vHv, void* stream) {
    clear_error();
    const State* s = reinterpret_cast<const State*>(state);
    if (!s || !in || !out) {
        set_error("null state or vector");
        return PQ_EINVAL;
    }
    if (in == out) {
        set_error("in and out must not overlap");
        return PQ_EINVAL;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    pq_status rc = apply_H_launch(*s, in, out, precision, nullptr, nullptr, 0, st);
    if (rc) return rc;
    if (out_vHv) {
        const int G = grid_size();
        if (precision == PQ_FP64)
            k_vhv_partials<double2><<<G, kVhvThreads, 0, st>>>((const double2*)in, (const double2*)out,
                                                               s->cnt + CNT_NA, (int64_t)s->cap, s->red_tmp);
        else
            k_vhv_partials<float2><<<G, kVhvThreads, 0, st>>>((const float2*)in, (const float2*)out,
                                                              s->cnt + CNT_NA, (int64_t)s->cap, s->red_tmp);
        PQ_CHECK_LAUNCH();
        k_vhv_sum<<<1, 32, 0, st>>>(s->red_tmp, G, out_vHv);
        PQ_CHECK_LAUNCH();
    }
#ifdef PQ_BOUNDS_CHECK
    // self-checking build: report a recorded out-of-range access at once
    return check_capacity(const_cast<State&>(*s), st);
#else
    return PQ_OK;
#endif
}

PQ_API pq_status pq_apply_H_host(pq_state* state, const void* in, void* out, int precision,
                                 void* stream) {
    clear_error();
    State* s = reinterpret_cast<State*>(state);
    if (!s || !in || !out) {
        set_error("null state or vector");
        return PQ_EINVAL;
    }
    if (precision != PQ_FP64 && precision != PQ_FP32MIX) {
        set_error("unknown precision %d", precision);
        return PQ_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!s->io_in) {
        pq_status rc;
        if ((rc = dalloc(&s->io_in, s->cap * 16)) || (rc = dalloc(&s->io_out, s->cap * 16)))
            return rc;
    }
    PQ_CUDA_TRY(cudaMemcpyAsync(s->h_cnt, s->cnt, CNT_SIZE * 8, cudaMemcpyDeviceToHost, st));
    PQ_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t n = std::min<int64_t>(s->h_cnt[CNT_NA], (int64_t)s->cap);
    const size_t bytes = (size_t)n * (precision == PQ_FP64 ? 16 : 8);
    if (n > 0) PQ_CUDA_TRY(cudaMemcpyAsync(s->io_in, in, bytes, cudaMemcpyHostToDevice, st));
    pq_status rc = apply_H_launch(*s, s->io_in, s->io_out, precision, nullptr, nullptr, 0, st);
    if (rc) return rc;
    if (n > 0) PQ_CUDA_TRY(cudaMemcpyAsync(out, s->io_out, bytes, cudaMemcpyDeviceToHost, st));
    PQ_CUDA_TRY(cudaStreamSynchronize(st));
    return PQ_OK;
}

PQ_API pq_status pq_prune(pq_state* state, double theta, int radius, double rel_excl,
                          void* stream) {
    clear_error();
    State* s = reinterpret_cast<State*>(state);
    if (!s || !(theta >= 0) || !std::isfinite(theta)) {
        set_error("bad state or theta");
        return PQ_EINVAL;
    }
    return prune_launch(*s, theta, radius, rel_excl, (cudaStream_t)stream);
}

PQ_API pq_status pq_propagate(pq_state* state, const pq_prop_desc* desc, int nsteps,
                              void* stream) {
    clear_error();
    State* s = reinterpret_cast<State*>(state);
    if (!s || !desc) {
        set_error("null state or descriptor");
        return PQ_EINVAL;
    }
    s->theta = desc->theta;
    if (s->pvb) return pvb_propagate(*s, *desc, nsteps, (cudaStream_t)stream);
    return propagate_impl(*s, *desc, nsteps, (cudaStream_t)stream);
}

PQ_API pq_status pq_observables_get(pq_state* state, pq_observables* out) {
    clear_error();
    State* s = reinterpret_cast<State*>(state);
    if (!s || !out) {
        set_error("null argument");
        return PQ_EINVAL;
    }
    if (s->obs_energy_pending && !s->obs.empty()) {
        double E = 0.0;
        pq_status rc = energy_of_current(*s, &E, 0);
        if (rc) return rc;
        s->obs.back().energy = E;
        s->obs_energy_pending = false;
    }
    const int64_t n = (int64_t)s->obs.size();
    if (out->count) *out->count = n;
    const int64_t m = std::min<int64_t>(n, out->capacity);
    for (int64_t i = 0; i < m; ++i) {
        const ObsRecord& o = s->obs[i];
        if (out->t) out->t[i] = o.t;
        if (out->c_re) out->c_re[i] = o.c_re;
        if (out->c_im) out->c_im[i] = o.c_im;
        if (out->norm2) out->norm2[i] = o.norm2;
        if (out->energy) out->energy[i] = o.energy;
        if (out->n_active) out->n_active[i] = o.n_active;
        if (out->n_wasted) out->n_wasted[i] = o.n_wasted;
    }
    return PQ_OK;
}

PQ_API pq_status pq_set_timing(pq_state* state, int enable) {
    clear_error();
    State* s = reinterpret_cast<State*>(state);
    if (!s) {
        set_error("null state");
        return PQ_EINVAL;
    }
    s->timing.enabled = enable != 0;
    s->timing.ms = 0;
    s->timing.n_apply = 0;
    s->timing.coef = 0;
    return PQ_OK;
}

PQ_API pq_status pq_timing_get(pq_state* state, double* apply_ms, int64_t* n_apply,
                               double* coef_applied) {
    clear_error();
    State* s = reinterpret_cast<State*>(state);
    if (!s) {
        set_error("null state");
        return PQ_EINVAL;
    }
    if (apply_ms) *apply_ms = s->timing.ms;
    if (n_apply) *n_apply = s->timing.n_apply;
    if (coef_applied) *coef_applied = s->timing.coef;
    return PQ_OK;
}
