// Adjoint gradient of the survival probability P = |<Psi(0)|Psi(T)>|^2 of a
// pruned propagation (not a construction of the paper, which computes only
// the autocorrelation, Eq. acorr; the gradient is taken of that quantity).
//
// On the recorded sequence of active sets A_0..A_N the propagation is linear,
//   psi_{n+1} = R_n U_n psi_n,  U_n = exp(-i H_{A_n} dt)  (SIL, Sec. 3.1),
// with R_n carrying coefficients from A_n to A_{n+1}.  With the adjoint kets
//   lambda_N = a0 on A_N,   lambda_n = U_n^dagger R_n^T lambda_{n+1},
// C = <a0|psi_N> has
//   dC/dtheta = <d a0|psi_N> + <lambda_0|d psi_0>
//             - i sum_n int_0^dt <U_n(dt-s)^dagger R_n^T lambda_{n+1}| dH/dtheta |U_n(s) psi_n> ds,
// the s-integral by Gauss-Legendre, every exponential by SIL (negative times
// for the adjoint), and dP/dtheta = 2 Re(conj(C) dC/dtheta).  psi_n is
// recomputed segment by segment from checkpoints taken every `ckpt` steps.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "device_util.cuh"

namespace pq {

constexpr int kAdjThreads = 256;
constexpr int kMaxParams = 16;

// n-point Gauss-Legendre rule on [-1, 1]: Newton iteration on P_n from the
// Chebyshev-like initial guesses, P_n by its three-term recurrence.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Per parameter p: sum_I conj(lam_I) dV_p(x_I) psi_I, with dV_p = sum_t c_t
// prod_k f_tk(i_k) over the parameter's terms [toff[p], toff[p+1]).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_grad_dots(
    const uint32_t* __restrict__ keys, const typename Cx<R>::T* __restrict__ lam,
    const typename Cx<R>::T* __restrict__ psi, const int64_t* na, int64_t cap, Lattice L,
    const double* __restrict__ tab, const double* __restrict__ coef, const int* __restrict__ toff,
    int np, double* partials) {
    const int64_t n = min(*na, cap);
    double acc[2 * kMaxParams];
    for (int i = 0; i < 2 * kMaxParams; ++i) acc[i] = 0.0;
    int d[kMaxD];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = keys[p];
        for (int k = 0; k < L.D; ++k) d[k] = (int)((key / L.stride[k]) % (uint32_t)L.n[k]);
        const auto a = lam[p];
        const auto b = psi[p];
        const double re = (double)a.x * b.x + (double)a.y * b.y;   // conj(a) b
        const double im = (double)a.x * b.y - (double)a.y * b.x;
        for (int q = 0; q < np; ++q) {
            double dv = 0.0;
            for (int t = toff[q]; t < toff[q + 1]; ++t) {
                double f = coef[t];
                for (int k = 0; k < L.D; ++k) f *= tab[((size_t)t * L.D + k) * kMaxN + d[k]];
                dv += f;
            }
            acc[2 * q] += dv * re;
            acc[2 * q + 1] += dv * im;
        }
    }
    __shared__ double sh[kAdjThreads / 32];
    for (int j = 0; j < 2 * np; ++j) {
        const double v = warp_sum(acc[j]);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kAdjThreads / 32; ++w) s += sh[w];
            partials[(size_t)blockIdx.x * 2 * np + j] = s;
        }
        __syncthreads();
    }
}

// Per entry q: sum_I conj(da_q(I)) x_I with da_q = a0 (mode -1) or the
// derivative of a0 with respect to the packet centre of internal mode m:
// df_m(i_m) prod_{k != m} f_k(i_k).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_packet_dots(
    const uint32_t* __restrict__ keys, const typename Cx<R>::T* __restrict__ x, const int64_t* na,
    int64_t cap, Lattice L, const double2* __restrict__ fac, const double2* __restrict__ dfac,
    const int* __restrict__ modes, int nq, double* partials) {
    const int64_t n = min(*na, cap);
    double acc[2 * (kMaxParams + 1)];
    for (int i = 0; i < 2 * (kMaxParams + 1); ++i) acc[i] = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = keys[p];
        const auto v = x[p];
        for (int q = 0; q < nq; ++q) {
            double ar = 1.0, ai = 0.0;
            for (int k = 0; k < L.D; ++k) {
                const int dk = (int)((key / L.stride[k]) % (uint32_t)L.n[k]);
                const double2 f = k == modes[q] ? dfac[k * kMaxN + dk] : fac[k * kMaxN + dk];
                const double nr = ar * f.x - ai * f.y, ni = ar * f.y + ai * f.x;
                ar = nr;
                ai = ni;
            }
            acc[2 * q] += ar * v.x + ai * v.y;        // conj(a) v
            acc[2 * q + 1] += ar * v.y - ai * v.x;
        }
    }
    __shared__ double sh[kAdjThreads / 32];
    for (int j = 0; j < 2 * nq; ++j) {
        const double v = warp_sum(acc[j]);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kAdjThreads / 32; ++w) s += sh[w];
            partials[(size_t)blockIdx.x * 2 * nq + j] = s;
        }
        __syncthreads();
    }
}

// FP32 coefficients widened exactly to FP64.
__global__ void k_widen(const float2* __restrict__ x, double2* __restrict__ y, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        y[p] = make_double2((double)x[p].x, (double)x[p].y);
}

namespace {

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) {
            cudaDeviceSynchronize();   // the gradient's kernels may still use it
            dev_free(p, 0, false);
        }
    }
};

pq_status dmalloc(DevBuf& b, size_t bytes) {
    b.p = dev_alloc(bytes, 0, false);
    if (!b.p) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed", bytes);
        return PQ_ENOMEM;
    }
    return PQ_OK;
}

// Sum of block partials [G][width] in block order, on the host.
pq_status read_sums(const void* dpart, int G, int width, std::vector<double>& out, cudaStream_t st) {
    std::vector<double> h((size_t)G * width);
    PQ_CUDA_TRY(cudaMemcpyAsync(h.data(), dpart, h.size() * 8, cudaMemcpyDeviceToHost, st));
    PQ_CUDA_TRY(cudaStreamSynchronize(st));
    out.assign(width, 0.0);
    for (int b = 0; b < G; ++b)
        for (int j = 0; j < width; ++j) out[j] += h[(size_t)b * width + j];
    return PQ_OK;
}

}  // namespace

pq_status survival_grad(State& s, const pq_prop_desc& d, int nsteps, int ckpt,
                        const pq_param_desc* params, int np, double* grad, double* P_out,
                        cudaStream_t st) {
    const Basis& b = *s.basis;
    const Lattice& L = s.lat;
    const int lv = s.lead_virtual, D = L.D;
    if (s.generic) {
        set_error("the adjoint gradient is provided for DVR bases only");
        return PQ_ENOTSUP;
    }
    if (np < 0 || np > kMaxParams || (np > 0 && (!params || !grad)) || nsteps < 1 || ckpt < 1 ||
        d.K < 1 || d.K > kMaxK || !(d.dt > 0) || !(d.theta >= 0)) {
        set_error("bad gradient request (nparams <= %d, nsteps >= 1, ckpt >= 1, K, dt, theta)",
                  kMaxParams);
        return PQ_EINVAL;
    }
    {
        pq_status nrc = check_neighbour_rule(s.lat, d.radius);
        if (nrc) return nrc;
    }
    if (d.integrator != PQ_SIL || d.sil_tol != 0.0) {
        // an error-controlled order makes each step depend on the state: the
        // forward map is then not linear on the frozen sets
        set_error("the adjoint gradient provides fixed-order SIL only");
        return PQ_ENOTSUP;
    }
    // ---- parameter tables
    std::vector<double> tab, coef;
    std::vector<int> toff(1, 0), pot_idx, cen_idx, cen_mode;
    for (int q = 0; q < np; ++q) {
        const pq_param_desc& pd = params[q];
        if (pd.kind == PQ_PARAM_CENTRE) {
            if (pd.mode < 0 || pd.mode >= b.D_user) {
                set_error("parameter %d: packet mode %d out of range", q, pd.mode);
                return PQ_EINVAL;
            }
            cen_idx.push_back(q);
            cen_mode.push_back(pd.mode + lv);
            continue;
        }
        if (pd.kind != PQ_PARAM_POTENTIAL || pd.nterms < 0 || (pd.nterms > 0 && !pd.dterms)) {
            set_error("parameter %d: unknown kind or missing terms", q);
            return PQ_EINVAL;
        }
        for (int t = 0; t < pd.nterms; ++t) {
            const pq_sop_term& tm = pd.dterms[t];
            if (!tm.factors || !std::isfinite(tm.coef)) {
                set_error("parameter %d term %d: no factors or bad coefficient", q, t);
                return PQ_EINVAL;
            }
            coef.push_back(tm.coef);
            for (int k = 0; k < D; ++k) {
                const int ku = k - lv;
                for (int i = 0; i < kMaxN; ++i) {
                    double v = 1.0;
                    if (ku >= 0 && tm.factors[ku].kind == PQ_FACTOR_DIAG) {
                        if (!tm.factors[ku].values) {
                            set_error("parameter %d term %d: diagonal factor without values", q, t);
                            return PQ_EINVAL;
                        }
                        v = i < b.modes[ku].n ? tm.factors[ku].values[i] : 0.0;
                    } else if (ku >= 0 && tm.factors[ku].kind != PQ_FACTOR_IDENTITY) {
                        set_error("parameter %d term %d: dH/dtheta must be diagonal in the DVR", q, t);
                        return PQ_ENOTSUP;
                    }
                    tab.push_back(v);
                }
            }
        }
        toff.push_back((int)coef.size());
        pot_idx.push_back(q);
    }
    // derivative packet factors: f = u/|u|, u_i = sqrt(w_i) g(x_i; q0);
    // du/dq0 = u ((x - q0)/(2 s^2) - i p0); df = du/|u| - u Re<u, du>/|u|^3
    std::vector<double> dfac((size_t)D * kMaxN * 2, 0.0);
    for (int ku = 0; ku < b.D_user; ++ku) {
        const int n = b.modes[ku].n;
        const double s2 = s.width[ku] * s.width[ku];
        const double amp = pow(2.0 * M_PI * s2, -0.25);
        std::vector<std::complex<double>> u(n), du(n);
        double nrm2 = 0.0, red = 0.0;
        for (int i = 0; i < n; ++i) {
            const double dx = b.x[ku][i] - s.q0[ku];
            const std::complex<double> g =
                amp * std::exp(std::complex<double>(-dx * dx / (4.0 * s2), s.p0[ku] * dx));
            u[i] = sqrt(b.w[ku][i]) * g;
            du[i] = u[i] * std::complex<double>(dx / (2.0 * s2), -s.p0[ku]);
            nrm2 += std::norm(u[i]);
            red += std::real(std::conj(u[i]) * du[i]);
        }
        const double nrm = sqrt(nrm2);
        for (int i = 0; i < n; ++i) {
            const std::complex<double> df = du[i] / nrm - u[i] * red / (nrm2 * nrm);
            dfac[((size_t)(ku + lv) * kMaxN + i) * 2] = df.real();
            dfac[((size_t)(ku + lv) * kMaxN + i) * 2 + 1] = df.imag();
        }
    }
    const int npot = (int)pot_idx.size(), ncen = (int)cen_idx.size();
    DevBuf d_tab, d_coef, d_toff, d_dfac, d_modes, d_part;
    const int G = grid_size() * 2;
    pq_status rc;
    if ((rc = dmalloc(d_tab, tab.size() * 8)) || (rc = dmalloc(d_coef, coef.size() * 8)) ||
        (rc = dmalloc(d_toff, toff.size() * 4)) || (rc = dmalloc(d_dfac, dfac.size() * 8)) ||
        (rc = dmalloc(d_modes, (ncen + 1) * 4)) ||
        (rc = dmalloc(d_part, (size_t)G * 2 * (kMaxParams + 1) * 8)))
        return rc;
    std::vector<int> qmodes(1, -1);   // entry 0: a0 itself (C), then the centres
    for (int m : cen_mode) qmodes.push_back(m);
    PQ_CUDA_TRY(cudaMemcpy(d_tab.p, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice));
    PQ_CUDA_TRY(cudaMemcpy(d_coef.p, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice));
    PQ_CUDA_TRY(cudaMemcpy(d_toff.p, toff.data(), toff.size() * 4, cudaMemcpyHostToDevice));
    PQ_CUDA_TRY(cudaMemcpy(d_dfac.p, dfac.data(), dfac.size() * 8, cudaMemcpyHostToDevice));
    PQ_CUDA_TRY(cudaMemcpy(d_modes.p, qmodes.data(), qmodes.size() * 4, cudaMemcpyHostToDevice));
    if ((rc = ensure_krylov(s, d.K))) return rc;

    const size_t esz = s.esize;
    auto count = [&](int64_t* n) -> pq_status {
        PQ_CUDA_TRY(cudaMemcpyAsync(s.h_cnt, s.cnt, CNT_SIZE * 8, cudaMemcpyDeviceToHost, st));
        PQ_CUDA_TRY(cudaStreamSynchronize(st));
        if (s.h_cnt[CNT_ERR] & 1) {
            set_error("active set outgrew the capacity during the gradient run");
            return PQ_ECAPACITY;
        }
        *n = std::min<int64_t>(s.h_cnt[CNT_NA], (int64_t)s.cap);
        return PQ_OK;
    };
    auto packet_dots_on = [&](const State& S, const void* x,
                              std::vector<std::complex<double>>& out) -> pq_status {
        const int nq = 1 + ncen;
        if (S.prec == PQ_FP64)
            k_packet_dots<double><<<G, kAdjThreads, 0, st>>>(
                S.keys, (const double2*)x, S.cnt + CNT_NA, (int64_t)S.cap, L, (const double2*)S.fac64,
                (const double2*)d_dfac.p, (const int*)d_modes.p, nq, (double*)d_part.p);
        else
            k_packet_dots<float><<<G, kAdjThreads, 0, st>>>(
                S.keys, (const float2*)x, S.cnt + CNT_NA, (int64_t)S.cap, L, (const double2*)S.fac64,
                (const double2*)d_dfac.p, (const int*)d_modes.p, nq, (double*)d_part.p);
        PQ_CHECK_LAUNCH();
        std::vector<double> h;
        pq_status r = read_sums(d_part.p, G, 2 * nq, h, st);
        if (r) return r;
        out.resize(nq);
        for (int q = 0; q < nq; ++q) out[q] = std::complex<double>(h[2 * q], h[2 * q + 1]);
        return PQ_OK;
    };
    auto copy = [&](void* dst, const void* src, int64_t n) -> pq_status {
        if (n > 0) PQ_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)n * esz, cudaMemcpyDeviceToDevice, st));
        return PQ_OK;
    };

    // ---- forward run, recording the sets and checkpoints
    if ((rc = init_bits_from_packet(s, s.theta, st)) || (rc = set_psi_from_packet(s, st))) return rc;
    std::vector<DevBuf> sets(nsteps + 1);
    std::vector<int64_t> na(nsteps + 1);
    const int nseg = (nsteps + ckpt - 1) / ckpt;
    std::vector<DevBuf> ck(nseg);
    auto record = [&](int n) -> pq_status {
        pq_status r = count(&na[n]);
        if (r) return r;
        if ((r = dmalloc(sets[n], (size_t)na[n] * 4))) return r;
        if (na[n] > 0)
            PQ_CUDA_TRY(cudaMemcpyAsync(sets[n].p, s.keys, (size_t)na[n] * 4,
                                        cudaMemcpyDeviceToDevice, st));
        if (n % ckpt == 0 && n < nsteps) {
            if ((r = dmalloc(ck[n / ckpt], (size_t)na[n] * esz))) return r;
            if ((r = copy(ck[n / ckpt].p, s.psi, na[n]))) return r;
        }
        return PQ_OK;
    };
    if ((rc = record(0))) return rc;
    for (int n = 0; n < nsteps; ++n) {
        if ((rc = sil_only(s, d, st)) || (rc = prune_launch(s, d.theta, d.radius, d.rel_excl, st)) ||
            (rc = record(n + 1)))
            return rc;
    }
    std::vector<std::complex<double>> pd;
    if ((rc = packet_dots_on(s, s.psi, pd))) return rc;
    const std::complex<double> C = pd[0];
    std::vector<std::complex<double>> dC(np, 0.0);
    for (int c = 0; c < ncen; ++c) dC[cen_idx[c]] += pd[1 + c];   // <d a0 | psi_N>

    // ---- backward sweep.  An FP32 forward run's sweep runs on an FP64 twin of
    // the state (same basis, capacity and packet): the recorded sets are the
    // FP32 run's, its checkpoints are widened exactly, and the adjoint kets,
    // the recomputed kets and the Gauss-Legendre integrands are FP64.  The
    // products of P's gradient over the integral have no FP32 cancellation
    // floor, while P, C and the sets are those of the FP32 forward run.
    struct Twin {
        State* t = nullptr;
        ~Twin() {
            if (t) free_twin(t);
        }
    } twin;
    const bool widen = s.prec != PQ_FP64;
    if (widen && (rc = make_fp64_twin(s, &twin.t))) return rc;
    State& B = widen ? *twin.t : s;
    const size_t besz = B.esize;
    if ((rc = ensure_krylov(B, d.K))) return rc;
    auto bcopy = [&](void* dst, const void* src, int64_t n) -> pq_status {
        if (n > 0) PQ_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)n * besz, cudaMemcpyDeviceToDevice, st));
        return PQ_OK;
    };
    // checkpoint (forward precision) -> B's coefficients
    auto restore = [&](void* dst, const void* ckp, int64_t n) -> pq_status {
        if (n <= 0) return PQ_OK;
        if (!widen) return bcopy(dst, ckp, n);
        k_widen<<<G * 4, kAdjThreads, 0, st>>>((const float2*)ckp, (double2*)dst, n);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    };
    DevBuf lam_b, mu_b, psig_b, seg_b;
    size_t vmax = 0;
    for (int64_t v : na) vmax = std::max<size_t>(vmax, (size_t)v);
    if ((rc = dmalloc(lam_b, vmax * besz)) || (rc = dmalloc(mu_b, vmax * besz)) ||
        (rc = dmalloc(psig_b, vmax * besz)) || (rc = dmalloc(seg_b, (size_t)ckpt * vmax * besz)))
        return rc;
    std::vector<double> gx, gw;
    gauss_legendre(5, gx, gw);
    // lambda_N = a0 on A_N
    if ((widen && (rc = load_set(B, (const uint32_t*)sets[nsteps].p, na[nsteps], st))) ||
        (rc = set_psi_from_packet(B, st)))
        return rc;
    pq_prop_desc dd = d;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int c = sg * ckpt, e = std::min(nsteps, c + ckpt);
        if ((rc = bcopy(lam_b.p, B.psi, na[e]))) return rc;
        // recompute psi_c .. psi_{e-1} on their recorded sets
        if ((rc = load_set(B, (const uint32_t*)sets[c].p, na[c], st)) ||
            (rc = restore(B.psi, ck[sg].p, na[c])))
            return rc;
        for (int n = c; n < e; ++n) {
            if ((rc = bcopy((char*)seg_b.p + (size_t)(n - c) * vmax * besz, B.psi, na[n]))) return rc;
            if (n + 1 < e) {
                dd.dt = d.dt;
                if ((rc = sil_only(B, dd, st)) ||
                    (rc = load_set(B, (const uint32_t*)sets[n + 1].p, na[n + 1], st, true)))
                    return rc;
            }
        }
        if ((rc = load_set(B, (const uint32_t*)sets[e].p, na[e], st)) || (rc = bcopy(B.psi, lam_b.p, na[e])))
            return rc;
        for (int n = e - 1; n >= c; --n) {
            // mu = R_n^T lambda_{n+1} on A_n
            if ((rc = load_set(B, (const uint32_t*)sets[n].p, na[n], st, true)) ||
                (rc = bcopy(mu_b.p, B.psi, na[n])))
                return rc;
            const void* psin = (char*)seg_b.p + (size_t)(n - c) * vmax * besz;
            for (size_t g = 0; g < gx.size() && npot > 0; ++g) {
                const double sgn = d.dt * (1.0 + gx[g]) / 2.0, wg = gw[g] * d.dt / 2.0;
                dd.dt = sgn;                                   // U(s) psi_n
                if ((rc = bcopy(B.psi, psin, na[n])) || (rc = sil_only(B, dd, st)) ||
                    (rc = bcopy(psig_b.p, B.psi, na[n])))
                    return rc;
                dd.dt = -(d.dt - sgn);                         // U(dt-s)^dagger mu
                if ((rc = bcopy(B.psi, mu_b.p, na[n])) || (rc = sil_only(B, dd, st))) return rc;
                if (B.prec == PQ_FP64)
                    k_grad_dots<double><<<G, kAdjThreads, 0, st>>>(
                        B.keys, (const double2*)B.psi, (const double2*)psig_b.p, B.cnt + CNT_NA,
                        (int64_t)B.cap, L, (const double*)d_tab.p, (const double*)d_coef.p,
                        (const int*)d_toff.p, npot, (double*)d_part.p);
                else
                    k_grad_dots<float><<<G, kAdjThreads, 0, st>>>(
                        B.keys, (const float2*)B.psi, (const float2*)psig_b.p, B.cnt + CNT_NA,
                        (int64_t)B.cap, L, (const double*)d_tab.p, (const double*)d_coef.p,
                        (const int*)d_toff.p, npot, (double*)d_part.p);
                PQ_CHECK_LAUNCH();
                std::vector<double> h;
                if ((rc = read_sums(d_part.p, G, 2 * npot, h, st))) return rc;
                for (int q = 0; q < npot; ++q)
                    dC[pot_idx[q]] += std::complex<double>(0.0, -wg) * std::complex<double>(h[2 * q], h[2 * q + 1]);
            }
            dd.dt = -d.dt;                                     // lambda_n = U^dagger mu
            if ((rc = bcopy(B.psi, mu_b.p, na[n])) || (rc = sil_only(B, dd, st))) return rc;
        }
    }
    // <lambda_0 | d psi_0> for the packet centres (psi_0 = a0 on A_0)
    if (ncen > 0) {
        if ((rc = packet_dots_on(B, B.psi, pd))) return rc;
        for (int c = 0; c < ncen; ++c) dC[cen_idx[c]] += std::conj(pd[1 + c]);
    }
    for (int q = 0; q < np; ++q) grad[q] = 2.0 * std::real(std::conj(C) * dC[q]);
    if (P_out) *P_out = std::norm(C);
    // leave the state at its initial packet
    if ((rc = init_bits_from_packet(s, s.theta, st)) || (rc = set_psi_from_packet(s, st))) return rc;
    PQ_CUDA_TRY(cudaStreamSynchronize(st));
    return PQ_OK;
}

}  // namespace pq

using namespace pq;

extern "C" __attribute__((visibility("default"))) pq_status pq_survival_grad(
    pq_state* state, const pq_prop_desc* desc, int nsteps, int ckpt_every,
    const pq_param_desc* params, int nparams, double* grad_out, double* P_out, void* stream) {
    clear_error();
    State* s = reinterpret_cast<State*>(state);
    if (!s || !desc) {
        set_error("null state or descriptor");
        return PQ_EINVAL;
    }
    return survival_grad(*s, *desc, nsteps, ckpt_every, params, nparams, grad_out, P_out,
                         (cudaStream_t)stream);
}
