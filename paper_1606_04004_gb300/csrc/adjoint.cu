// Adjoint gradient of the survival probability P = |<Psi(0)|Psi(T)>|^2 of a
// pruned propagation (not a construction of the paper, which computes only
// the autocorrelation, Eq. acorr; the gradient is taken of that quantity).
//
// On the recorded sequence of active sets A_0..A_N the propagation is
//   psi_{n+1} = R_n S_n(psi_n),  S_n = the fixed-order SIL step on A_n (Sec. 3.1),
// with R_n carrying coefficients from A_n to A_{n+1} (kept where the point
// stays, zero where it is new).  The gradient is that of this discrete map, so
// it agrees with finite differences of the propagation whether or not the SIL
// step has converged to exp(-i H dt): with dL = Re<xbar, dx> for every ket x,
//   psibar_N = 2 C a0 on A_N,  psibar_n = S_n'(psi_n)^dagger R_n^T psibar_{n+1},
// where the reverse pass through S_n repeats the step's Lanczos recurrence and
// runs it backwards (its scalars on the host, its vectors on the device); the
// potential parameters collect Re<wbar_k, dH/dtheta V_k> at every Lanczos
// vector, the packet centres Re<psibar_0, d a0> plus the bra's share
// 2 Re(conj(C) <d a0|psi_N>).  psi_n is recomputed segment by segment from
// checkpoints taken every `ckpt` steps.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "device_util.cuh"

namespace pq {

constexpr int kAdjThreads = 256;
constexpr int kMaxParams = 16;

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

// ---------------------------------------------- the step's discrete adjoint
// Vector primitives of the reverse sweep through one Lanczos step (FP64
// kets, at most kChunk vectors per launch, Krylov vectors ld elements apart).
constexpr int kChunk = 8;
struct Coefs {
    double2 c[kMaxK + 1];
};

// partials[b][2m] = block sums of <V_i, x> = sum_I conj(V_i,I) x_I, i < m.
__global__ void __launch_bounds__(kAdjThreads) k_mdot(const double2* __restrict__ V, size_t ld,
                                                      int m, const double2* __restrict__ x,
                                                      const int64_t* na, int64_t cap,
                                                      double* partials) {
    const int64_t n = min(*na, cap);
    double acc[2 * kChunk];
#pragma unroll
    for (int i = 0; i < 2 * kChunk; ++i) acc[i] = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double2 b = x[p];
#pragma unroll
        for (int i = 0; i < kChunk; ++i) {
            if (i < m) {
                const double2 a = V[(size_t)i * ld + p];
                acc[2 * i] += a.x * b.x + a.y * b.y;
                acc[2 * i + 1] += a.x * b.y - a.y * b.x;
            }
        }
    }
    __shared__ double sh[kAdjThreads / 32];
    for (int j = 0; j < 2 * m; ++j) {
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < 2 * kChunk; ++i)
            if (i == j) v = acc[i];
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kAdjThreads / 32; ++w) s += sh[w];
            partials[(size_t)blockIdx.x * 2 * m + j] = s;
        }
        __syncthreads();
    }
}

// out = sx x + sum_{i<m} c_i V_i  (x nullable; out may be x, not a V_i).
__global__ void k_mcomb(double2* out, const double2* x, double2 sx, const double2* __restrict__ V,
                        size_t ld, int m, Coefs cf, const int64_t* na, int64_t cap) {
    const int64_t n = min(*na, cap);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        if (x) {
            const double2 v = x[p];
            re = sx.x * v.x - sx.y * v.y;
            im = sx.x * v.y + sx.y * v.x;
        }
        for (int i = 0; i < m; ++i) {
            const double2 v = V[(size_t)i * ld + p], c = cf.c[i];
            re += c.x * v.x - c.y * v.y;
            im += c.x * v.y + c.y * v.x;
        }
        out[p] = make_double2(re, im);
    }
}

// Y_i = (init ? 0 : Y_i) + c_i x for i < m (Y_i ld elements apart; x is no Y_i).
__global__ void k_mout(double2* Y, size_t ld, int m, const double2* __restrict__ x, Coefs cf,
                       int init, const int64_t* na, int64_t cap) {
    const int64_t n = min(*na, cap);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[p];
        for (int i = 0; i < m; ++i) {
            const double2 c = cf.c[i];
            double2* y = Y + (size_t)i * ld + p;
            const double2 o = init ? make_double2(0.0, 0.0) : *y;
            *y = make_double2(o.x + c.x * v.x - c.y * v.y, o.y + c.x * v.y + c.y * v.x);
        }
    }
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
        if (n % ckpt == 0 && n < nsteps && s.prec == PQ_FP64) {
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
    // the state (same basis, capacity and packet): the sets are the FP32 run's,
    // and the twin replays the propagation on them in FP64 from the initial
    // packet, keeping FP64 checkpoints, so that the recomputed kets, the
    // adjoint kets and the gradient sums are FP64 (the FP32 run's own states
    // carry its rounding, which P's strong curvature in lambda turns into a
    // gradient error above 1e-4).  P, C and the sets are those of the FP32
    // forward run.
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
    if (widen) {   // FP64 replay on the recorded sets: the checkpoints
        if ((rc = load_set(B, (const uint32_t*)sets[0].p, na[0], st)) || (rc = set_psi_from_packet(B, st)))
            return rc;
        for (int n = 0; n < nsteps; ++n) {
            if (n % ckpt == 0) {
                if ((rc = dmalloc(ck[n / ckpt], std::max<size_t>((size_t)na[n], 1) * besz)) ||
                    (rc = bcopy(ck[n / ckpt].p, B.psi, na[n])))
                    return rc;
            }
            if ((rc = sil_only(B, d, st)) ||
                (rc = load_set(B, (const uint32_t*)sets[n + 1].p, na[n + 1], st, true)))
                return rc;
        }
    }
    DevBuf lam_b, seg_b, vjp_b;
    size_t vmax = 0;
    for (int64_t v : na) vmax = std::max<size_t>(vmax, (size_t)v);
    vmax = std::max<size_t>(vmax, 1);
    const int K = d.K;
    // per step: V_0..V_{K-1}, W_k = H V_k, their cotangents, and wbar, ubar, H wbar
    if ((rc = dmalloc(lam_b, vmax * besz)) || (rc = dmalloc(seg_b, (size_t)ckpt * vmax * besz)) ||
        (rc = dmalloc(vjp_b, (size_t)(3 * K + 3) * vmax * 16)))
        return rc;
    double2* const Vv = (double2*)vjp_b.p;
    double2* const Wv = Vv + (size_t)K * vmax;
    double2* const Vb = Wv + (size_t)K * vmax;
    double2* const wb = Vb + (size_t)K * vmax;
    double2* const ub = wb + vmax;
    double2* const hw = ub + vmax;
    auto vk = [&](double2* base, int k) { return base + (size_t)k * vmax; };
    const int64_t* dna = B.cnt + CNT_NA;
    const int64_t bcap = (int64_t)B.cap;
    using cd = std::complex<double>;
    // <V_i, x> for i < m (V_i vmax elements apart)
    auto mdot = [&](const double2* V, int m, const double2* x, std::vector<cd>& out) -> pq_status {
        out.assign(m, 0.0);
        for (int i0 = 0; i0 < m; i0 += kChunk) {
            const int mm = std::min(kChunk, m - i0);
            k_mdot<<<G, kAdjThreads, 0, st>>>(V + (size_t)i0 * vmax, vmax, mm, x, dna, bcap,
                                             (double*)d_part.p);
            PQ_CHECK_LAUNCH();
            std::vector<double> h;
            pq_status r = read_sums(d_part.p, G, 2 * mm, h, st);
            if (r) return r;
            for (int i = 0; i < mm; ++i) out[i0 + i] = cd(h[2 * i], h[2 * i + 1]);
        }
        return PQ_OK;
    };
    // <v, x>; a failed reduction leaves its status in dot_rc and returns NaN,
    // which the finiteness checks below turn into an error
    pq_status dot_rc = PQ_OK;
    auto dot1 = [&](const double2* v, const double2* x) -> cd {
        std::vector<cd> o;
        const pq_status r = mdot(v, 1, x, o);
        if (r) {
            if (!dot_rc) dot_rc = r;
            return cd(NAN, NAN);
        }
        return o[0];
    };
    auto pack = [&](const std::vector<cd>& c, int i0, int m, cd scale, bool conjugate) {
        Coefs cf;
        for (int i = 0; i < m; ++i) {
            const cd v = scale * (conjugate ? std::conj(c[i0 + i]) : c[i0 + i]);
            cf.c[i] = make_double2(v.real(), v.imag());
        }
        return cf;
    };
    // out = sx x + sum_{i<m} c_i V_i
    auto mcomb = [&](double2* out, const double2* x, cd sx, const double2* V, int m,
                     const Coefs& cf) -> pq_status {
        k_mcomb<<<G * 4, kAdjThreads, 0, st>>>(out, x, make_double2(sx.real(), sx.imag()), V, vmax,
                                               m, cf, dna, bcap);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    };
    auto mout = [&](double2* Y, int m, const double2* x, const Coefs& cf, int init) -> pq_status {
        for (int i0 = 0; i0 < m; i0 += kChunk) {
            Coefs part;
            const int mm = std::min(kChunk, m - i0);
            for (int i = 0; i < mm; ++i) part.c[i] = cf.c[i0 + i];
            k_mout<<<G * 4, kAdjThreads, 0, st>>>(Y + (size_t)i0 * vmax, vmax, mm, x, part, init,
                                                  dna, bcap);
            PQ_CHECK_LAUNCH();
        }
        return PQ_OK;
    };
    auto Hx = [&](const double2* in, double2* out) -> pq_status {
        return apply_H_launch(B, in, out, PQ_FP64, nullptr, nullptr, 0, st);
    };
    std::vector<double> thbar(npot, 0.0);

    // Reverse pass through one SIL step on the current set of B (Sec. 3.1 with
    // the order fixed): on entry B.psi holds ybar, the cotangent of the step's
    // output (dL = Re<ybar, dy>); on exit it holds the cotangent of the input a,
    // and thbar has gained the step's Re<wbar_k, dH/dtheta V_k>.  The forward
    // Lanczos process is repeated in FP64 with explicitly normalised vectors and
    // one classical Gram-Schmidt pass against all previous vectors (equal, in
    // exact arithmetic, to the three-term recurrence of the propagation, so the
    // derivative is that of the same map):
    //   V_0 = a/b0, W_k = H V_k, c_ik = <V_i, W_k>, alpha_k = Re c_kk,
    //   u_k = W_k - sum_i c_ik V_i, beta_k = ||u_k||, V_{k+1} = u_k/beta_k,
    //   y = b0 sum_j e_j V_j,  e = exp(-i T dt) e_1 of the Lanczos tridiagonal T.
    // The derivative of e with respect to T is the Daleckii-Krein formula in T's
    // eigenbasis (divided differences of exp(-i z dt)).
    auto step_vjp = [&](const double2* a) -> pq_status {
        double2* ybar = (double2*)B.psi;
        const double n0 = dot1(a, a).real();
        if (dot_rc) return dot_rc;
        if (!std::isfinite(n0)) {
            set_error("non-finite state in the gradient's reverse sweep");
            return PQ_ENUMERIC;
        }
        const double b0 = sqrt(std::max(0.0, n0));
        if (!(b0 > 0.0)) return PQ_OK;   // zero state: the step is the identity
        const Coefs none{};
        pq_status r;
        if ((r = mcomb(vk(Vv, 0), a, 1.0 / b0, nullptr, 0, none))) return r;
        std::vector<std::vector<cd>> c(K);
        std::vector<double> alpha(K, 0.0), beta(K, 0.0);
        int Ke = K;
        for (int k = 0; k < K; ++k) {
            if ((r = Hx(vk(Vv, k), vk(Wv, k)))) return r;
            const int i0 = k == K - 1 ? k : 0;
            std::vector<cd> ck;
            if ((r = mdot(vk(Vv, i0), k - i0 + 1, vk(Wv, k), ck))) return r;
            c[k].assign(k + 1, 0.0);
            for (int i = i0; i <= k; ++i) c[k][i] = ck[i - i0];
            alpha[k] = c[k][k].real();
            if (k == K - 1) break;
            if ((r = mcomb(vk(Vv, k + 1), vk(Wv, k), 1.0, vk(Vv, 0), k + 1, pack(c[k], 0, k + 1, -1.0, false))))
                return r;
            const double b2 = dot1(vk(Vv, k + 1), vk(Vv, k + 1)).real();
            const double h2 = dot1(vk(Wv, k), vk(Wv, k)).real();
            if (dot_rc) return dot_rc;
            const double b = sqrt(std::max(0.0, b2)), hn = sqrt(std::max(0.0, h2));
            if (!std::isfinite(b2) || !std::isfinite(h2) || !std::isfinite(alpha[k])) {
                set_error("non-finite Lanczos scalars in the gradient's reverse sweep");
                return PQ_ENUMERIC;
            }
            if (b <= 1e-12 * hn) {   // invariant subspace: the propagation stops here too
                Ke = k + 1;
                break;
            }
            beta[k] = b;
            if ((r = mcomb(vk(Vv, k + 1), vk(Vv, k + 1), 1.0 / b, nullptr, 0, none))) return r;
        }
        // T = Z diag(lam) Z^T; e_j = sum_p Z_jp exp(-i lam_p dt) Z_0p
        std::vector<double> T((size_t)Ke * Ke, 0.0), lam, Z;
        for (int k = 0; k < Ke; ++k) {
            T[(size_t)k * Ke + k] = alpha[k];
            if (k + 1 < Ke) T[(size_t)k * Ke + k + 1] = T[(size_t)(k + 1) * Ke + k] = beta[k];
        }
        if (jacobi_eigh(Ke, T, lam, Z) < 0) {
            set_error("eigensolver of the Lanczos tridiagonal did not converge");
            return PQ_ENUMERIC;
        }
        auto z = [&](int i, int j) { return Z[(size_t)i * Ke + j]; };
        const double dt = d.dt;
        std::vector<cd> e(Ke, 0.0);
        for (int j = 0; j < Ke; ++j)
            for (int q = 0; q < Ke; ++q) e[j] += z(j, q) * std::exp(cd(0.0, -lam[q] * dt)) * z(0, q);
        // cotangents of e, b0 and the V_j from y = b0 sum_j e_j V_j
        std::vector<cd> ebar;
        if ((r = mdot(vk(Vv, 0), Ke, ybar, ebar))) return r;
        double b0bar = 0.0;
        for (int j = 0; j < Ke; ++j) {
            ebar[j] *= b0;
            b0bar += std::real(e[j] * std::conj(ebar[j]));
        }
        b0bar /= b0;
        {
            std::vector<cd> s(Ke);
            for (int j = 0; j < Ke; ++j) s[j] = b0 * std::conj(e[j]);
            if ((r = mout(Vb, Ke, ybar, pack(s, 0, Ke, 1.0, false), 1))) return r;
        }
        // Tbar = Z Re(Y o G) Z^T with Y_pq = sum_i Z_ip ebar_i Z_0q and G_pq the
        // divided difference of exp(+i z dt) at lam_p, lam_q
        std::vector<double> Tbar((size_t)Ke * Ke, 0.0), RY((size_t)Ke * Ke);
        for (int p = 0; p < Ke; ++p) {
            cd zp = 0.0;
            for (int i = 0; i < Ke; ++i) zp += z(i, p) * ebar[i];
            for (int q = 0; q < Ke; ++q) {
                const double x = dt * (lam[p] - lam[q]);
                const cd g = std::exp(cd(0.0, lam[q] * dt));
                const cd G = std::fabs(x) < 1e-8 ? cd(0.0, dt) * g * cd(1.0, 0.5 * x)
                                                 : g * (std::exp(cd(0.0, x)) - 1.0) / (lam[p] - lam[q]);
                RY[(size_t)p * Ke + q] = std::real(zp * z(0, q) * G);
            }
        }
        for (int i = 0; i < Ke; ++i)
            for (int j = 0; j < Ke; ++j) {
                double acc = 0.0;
                for (int p = 0; p < Ke; ++p)
                    for (int q = 0; q < Ke; ++q) acc += z(i, p) * RY[(size_t)p * Ke + q] * z(j, q);
                Tbar[(size_t)i * Ke + j] = acc;
            }
        // reverse Lanczos recurrence
        for (int k = Ke - 1; k >= 0; --k) {
            const bool last = k == Ke - 1;
            const int i0 = last ? k : 0;
            std::vector<cd> cbar(k + 1, 0.0);
            if (!last) {
                const double b = beta[k];
                const double rr = dot1(vk(Vv, k + 1), vk(Vb, k + 1)).real();
                if (dot_rc) return dot_rc;
                const double bebar = Tbar[(size_t)k * Ke + k + 1] + Tbar[(size_t)(k + 1) * Ke + k];
                Coefs cv{};
                cv.c[0] = make_double2(bebar - rr / b, 0.0);
                // ubar = Vbar_{k+1}/beta_k + (betabar_k - Re<V_{k+1}, Vbar_{k+1}>/beta_k) V_{k+1}
                if ((r = mcomb(ub, vk(Vb, k + 1), 1.0 / b, vk(Vv, k + 1), 1, cv))) return r;
                std::vector<cd> dv;
                if ((r = mdot(vk(Vv, 0), k + 1, ub, dv))) return r;
                for (int i = 0; i <= k; ++i) cbar[i] = -dv[i];
                if ((r = mout(Vb, k + 1, ub, pack(c[k], 0, k + 1, -1.0, true), 0))) return r;
            }
            cbar[k] += Tbar[(size_t)k * Ke + k];   // alpha_k = Re c_kk
            // wbar = ubar + sum_i cbar_i V_i ; Vbar_i += conj(cbar_i) W_k ; Vbar_k += H wbar
            if ((r = mcomb(wb, last ? nullptr : ub, 1.0, vk(Vv, i0), k - i0 + 1,
                           pack(cbar, i0, k - i0 + 1, 1.0, false))) ||
                (r = mout(vk(Vb, i0), k - i0 + 1, vk(Wv, k), pack(cbar, i0, k - i0 + 1, 1.0, true), 0)) ||
                (r = Hx(wb, hw)))
                return r;
            Coefs one{};
            one.c[0] = make_double2(1.0, 0.0);
            if ((r = mcomb(vk(Vb, k), vk(Vb, k), 1.0, hw, 1, one))) return r;
            if (npot > 0) {
                k_grad_dots<double><<<G, kAdjThreads, 0, st>>>(
                    B.keys, wb, vk(Vv, k), dna, bcap, L, (const double*)d_tab.p,
                    (const double*)d_coef.p, (const int*)d_toff.p, npot, (double*)d_part.p);
                PQ_CHECK_LAUNCH();
                std::vector<double> h;
                if ((r = read_sums(d_part.p, G, 2 * npot, h, st))) return r;
                for (int q = 0; q < npot; ++q) thbar[q] += h[2 * q];
            }
        }
        // abar = Vbar_0/b0 + (b0bar - Re<V_0, Vbar_0>/b0) V_0
        const double r0 = dot1(vk(Vv, 0), vk(Vb, 0)).real();
        if (dot_rc) return dot_rc;
        Coefs cv{};
        cv.c[0] = make_double2(b0bar - r0 / b0, 0.0);
        return mcomb((double2*)B.psi, vk(Vb, 0), 1.0 / b0, vk(Vv, 0), 1, cv);
    };

    // psibar_N = 2 C a0 on A_N  (dP = Re<psibar_N, d psi_N> + the bra's share)
    if ((widen && (rc = load_set(B, (const uint32_t*)sets[nsteps].p, na[nsteps], st))) ||
        (rc = set_psi_from_packet(B, st)))
        return rc;
    {
        const Coefs none{};
        if ((rc = mcomb((double2*)B.psi, (const double2*)B.psi, 2.0 * C, nullptr, 0, none))) return rc;
    }
    pq_prop_desc dd = d;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int c = sg * ckpt, e = std::min(nsteps, c + ckpt);
        if ((rc = bcopy(lam_b.p, B.psi, na[e]))) return rc;
        // recompute psi_c .. psi_{e-1} on their recorded sets
        if ((rc = load_set(B, (const uint32_t*)sets[c].p, na[c], st)) ||
            (rc = bcopy(B.psi, ck[sg].p, na[c])))
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
            // ybar = R_n^T psibar_{n+1} on A_n, then the step's reverse pass
            if ((rc = load_set(B, (const uint32_t*)sets[n].p, na[n], st, true)) ||
                (rc = step_vjp((const double2*)((char*)seg_b.p + (size_t)(n - c) * vmax * besz))))
                return rc;
        }
    }
    for (int q = 0; q < npot; ++q) grad[pot_idx[q]] = thbar[q];
    // packet centres: the bra's share 2 Re(conj(C) <d a0|psi_N>) and the
    // initial state's Re<psibar_0, d a0> (psi_0 = a0 on A_0)
    for (int cc = 0; cc < ncen; ++cc) grad[cen_idx[cc]] = 2.0 * std::real(std::conj(C) * dC[cen_idx[cc]]);
    if (ncen > 0) {
        if ((rc = packet_dots_on(B, B.psi, pd))) return rc;
        for (int cc = 0; cc < ncen; ++cc) grad[cen_idx[cc]] += std::real(pd[1 + cc]);
    }
    for (int q = 0; q < np; ++q)
        if (!std::isfinite(grad[q])) {
            set_error("non-finite gradient component %d", q);
            return PQ_ENUMERIC;
        }
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
