// Short-iterative Lanczos propagation on the device (Sec. 3.1: short
// iterative Arnoldi; for Hermitian H its Hessenberg matrix is the Lanczos
// tridiagonal), the adaption after every step (Sec. 2.5) and the observables
// (Eq. acorr).  All Lanczos scalars live on the device in FP64; the host never
// waits inside a step.
//
// Per step, with V_0 = psi (scale 1/beta_0) and the new Krylov vector written
// in place into its slot:
//   W = H V_k                               (apply_H, input scaled by sigma_k)
//   c_i = <V_i, W> for the vectors kept      (dots, FP64 or double-float sums)
//   W <- W - sum_i c_i V_i,  beta_k = ||W||  (update; sigma_{k+1} = 1/beta_k)
//   psi <- beta_0 V_K exp(-i T_K dt) e_1     (exp of the K x K tridiagonal)
// Reductions are deterministic: fixed-order per-block partials, then one
// block sums them in block order.
#include <math.h>

#include <algorithm>

#include "device_util.cuh"

namespace pq {

constexpr int kRedThreads = 256;
constexpr int kMaxM = 16;   // Krylov vectors handled per dots / update launch

static int red_blocks() { return grid_size() * 8; }

// accumulator: FP64 for double inputs, double-float for float inputs
template <typename R> struct Acc;
template <> struct Acc<double> {
    double v;
    __device__ void init() { v = 0.0; }
    __device__ void add(double x) { v += x; }
    __device__ double value() const { return v; }
};
template <> struct Acc<float> {
    DF v;
    __device__ void init() { v.hi = 0.f; v.lo = 0.f; }
    __device__ void add(float x) { df_add(v, x); }
    __device__ double value() const { return df_value(v); }
};

// Sum WIDTH per-thread doubles over the block (blockDim.x == kRedThreads);
// thread j < WIDTH writes sum j to partials[blockIdx.x * WIDTH + j].  Warp
// sums first, then one thread per value adds the warps in order.
template <int WIDTH>
__device__ __forceinline__ void block_partials(const double (&vals)[WIDTH], double* partials) {
    constexpr int kWarps = kRedThreads / 32;
    __shared__ double sh[WIDTH][kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < WIDTH; ++j) {
        const double v = warp_sum(vals[j]);
        if (lane == 0) sh[j][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < WIDTH) {
        double x = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) x += sh[threadIdx.x][w];
        partials[(size_t)blockIdx.x * WIDTH + threadIdx.x] = x;
    }
}

// Column sums of partials[G][width] -> out[width]: warp j sums column j
// with a fixed lane-strided order (four interleaved accumulators per lane, so
// that four loads are in flight) and a fixed butterfly (deterministic).
__device__ void sum_partials(const double* partials, int G, int width, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = wid; j < width; j += nw) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int b = lane;
        for (; b + 96 < G; b += 128) {
            const double x0 = partials[(size_t)b * width + j];
            const double x1 = partials[(size_t)(b + 32) * width + j];
            const double x2 = partials[(size_t)(b + 64) * width + j];
            const double x3 = partials[(size_t)(b + 96) * width + j];
            a0 += x0;
            a1 += x1;
            a2 += x2;
            a3 += x3;
        }
        for (; b < G; b += 32) a0 += partials[(size_t)b * width + j];
        double acc = (a0 + a1) + (a2 + a3);
        acc = warp_sum(acc);
        if (lane == 0) out[j] = acc;
    }
}

template <typename R>
__device__ __forceinline__ const typename Cx<R>::T* kvec(const void* psi, const void* Vb,
                                                          size_t cap, int i) {
    using V = typename Cx<R>::T;
    return i == 0 ? (const V*)psi : (const V*)Vb + (size_t)(i - 1) * cap;
}

// ---------------------------------------------------------------- norm
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_norm2(const typename Cx<R>::T* __restrict__ x,
                                                        const int64_t* na, int64_t cap,
                                                        double* partials) {
    const int64_t n = min(*na, cap);
    Acc<R> acc;
    acc.init();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const auto v = x[p];
        acc.add(v.x * v.x + v.y * v.y);
    }
    const double vals[1] = {acc.value()};
    block_partials<1>(vals, partials);
}

// beta_0 = ||psi||; sigma_0 = 1/beta_0; reset the step's scalars.  track
// (FP32-mix): the target norm of this step's output follows the adaption
// since the previous output (see k_renorm_factor).
__global__ void k_start_step(const double* partials, int G, KrylovScalars* ks, int K,
                             int64_t* err, int track = 0) {
    __shared__ double tot[1];
    sum_partials(partials, G, 1, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double n2 = tot[0];
        ks->keff = K;
        if (!(n2 > 0.0) || !isfinite(n2)) {
            // empty or zero state: nothing to propagate
            ks->beta0 = 0.0;
            ks->sigma[0] = 0.0;
            ks->keff = 0;
            if (!isfinite(n2)) *err |= 2;
        } else {
            ks->beta0 = sqrt(n2);
            ks->sigma[0] = 1.0 / ks->beta0;
        }
        if (track) {
            if (ks->rn_target > 0.0 && ks->rn_last > 0.0 && ks->beta0 > 0.0)
                ks->rn_target *= ks->beta0 / ks->rn_last;
            else
                ks->rn_target = ks->beta0;
        }
    }
}

// ---------------------------------------------------------------- dots
// c_i = sigma_i <V_i, W> for i in [i0, i0 + M) and ||W||^2.  Each thread takes
// two elements per iteration; their products are summed in R before entering
// the accumulator (double-float for FP32 data, FP64 for FP64 data).
template <typename R, int M>
__global__ void __launch_bounds__(kRedThreads) k_dots(const void* psi, const void* Vb, size_t cap,
                                                       const typename Cx<R>::T* __restrict__ W,
                                                       const int64_t* na, int i0,
                                                       const KrylovScalars* ks, int k,
                                                       double* partials) {
    if (ks->keff <= k) return;
    const int64_t n = min(*na, (int64_t)cap);
    Acc<R> ar[M], ai[M], an;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        ar[i].init();
        ai[i].init();
    }
    an.init();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += 2 * stride) {
        const int64_t q = p + stride;
        const bool has2 = q < n;
        const auto w = W[p];
        const auto w2 = has2 ? W[q] : cmake<R>(0, 0);
        typename Cx<R>::T v[M], v2[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const auto* vi = kvec<R>(psi, Vb, cap, i0 + i);
            v[i] = vi[p];
            v2[i] = has2 ? vi[q] : cmake<R>(0, 0);
        }
        an.add((w.x * w.x + w.y * w.y) + (w2.x * w2.x + w2.y * w2.y));
#pragma unroll
        for (int i = 0; i < M; ++i) {
            // conj(v) * w over both elements
            ar[i].add((v[i].x * w.x + v[i].y * w.y) + (v2[i].x * w2.x + v2[i].y * w2.y));
            ai[i].add((v[i].x * w.y - v[i].y * w.x) + (v2[i].x * w2.y - v2[i].y * w2.x));
        }
    }
    double vals[2 * M + 1];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        vals[2 * i] = ar[i].value();
        vals[2 * i + 1] = ai[i].value();
    }
    vals[2 * M] = an.value();
    block_partials<2 * M + 1>(vals, partials);
}

// Finalise the dots of step k: scale by sigma_i, store, record alpha_k.
// obs_prev (nullable): E of the previous record = alpha_0.
__global__ void k_dots_done(const double* partials, int G, int i0, int m, KrylovScalars* ks,
                            int k, double* obs_prev_E, int64_t* err) {
    __shared__ double tot[2 * kMaxM + 1];
    if (ks->keff <= k) return;
    sum_partials(partials, G, 2 * m + 1, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < m; ++i) {
            const double sg = ks->sigma[i0 + i];
            ks->dots[2 * (i0 + i)] = tot[2 * i] * sg;
            ks->dots[2 * (i0 + i) + 1] = tot[2 * i + 1] * sg;
        }
        if (i0 + m - 1 == k) {
            ks->alpha[k] = ks->dots[2 * k];
            ks->hnorm2 = tot[2 * m];
            if (!isfinite(ks->alpha[k])) *err |= 2;
            if (k == 0 && obs_prev_E) *obs_prev_E = ks->alpha[0];
        }
    }
}

// ---------------------------------------------------------------- update
// W <- W - sum_{i in [i0, i0+M)} c_i sigma_i V_i ; optional ||W||^2 partials.
template <typename R, int M>
__global__ void __launch_bounds__(kRedThreads) k_update(const void* psi, const void* Vb, size_t cap,
                                                         typename Cx<R>::T* __restrict__ W,
                                                         const int64_t* na, int i0,
                                                         const KrylovScalars* ks, int k,
                                                         int want_norm, double* partials) {
    if (ks->keff <= k) return;
    const int64_t n = min(*na, (int64_t)cap);
    R cr[M], ci[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const double sg = ks->sigma[i0 + i];
        cr[i] = (R)(ks->dots[2 * (i0 + i)] * sg);
        ci[i] = (R)(ks->dots[2 * (i0 + i) + 1] * sg);
    }
    Acc<R> an;
    an.init();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += 2 * stride) {
        const int64_t q = p + stride;
        const bool has2 = q < n;
        auto w = W[p];
        auto w2 = has2 ? W[q] : cmake<R>(0, 0);
        typename Cx<R>::T v[M], v2[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const auto* vi = kvec<R>(psi, Vb, cap, i0 + i);
            v[i] = vi[p];
            v2[i] = has2 ? vi[q] : cmake<R>(0, 0);
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            // w -= c * v  (c complex)
            w.x -= cr[i] * v[i].x - ci[i] * v[i].y;
            w.y -= cr[i] * v[i].y + ci[i] * v[i].x;
            w2.x -= cr[i] * v2[i].x - ci[i] * v2[i].y;
            w2.y -= cr[i] * v2[i].y + ci[i] * v2[i].x;
        }
        W[p] = w;
        if (has2) W[q] = w2;
        else w2 = cmake<R>(0, 0);
        if (want_norm) an.add((w.x * w.x + w.y * w.y) + (w2.x * w2.x + w2.y * w2.y));
    }
    if (want_norm) {
        const double vals[1] = {an.value()};
        block_partials<1>(vals, partials);
    }
}

// Grid of a grid-stride reduction kernel: at most G blocks, and no more than
// fit on the GPU at once (the kernel's occupancy x SMs), so that a launch is
// one full wave, with no partly filled second wave, and fewer partials to sum.
template <typename F>
static int one_wave_grid(F kernel, int G) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRedThreads, 0) !=
            cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();   // clear the query's error; keep the default grid
        return G;
    }
    return std::max(1, std::min(G, per_sm * grid_size()));
}

// Launch k_dots / k_update for a run-time count m in [1, kMaxM] on at most G
// blocks; returns the block count used (the row count of the partials).
template <typename R, int M = 1>
static int launch_dots(int m, int G, cudaStream_t st, const void* psi, const void* Vb,
                       size_t cap, const typename Cx<R>::T* W, const int64_t* na, int i0,
                       const KrylovScalars* ks, int k, double* partials) {
    if constexpr (M < kMaxM) {
        if (m != M) return launch_dots<R, M + 1>(m, G, st, psi, Vb, cap, W, na, i0, ks, k, partials);
    }
    static const int g = one_wave_grid(k_dots<R, M>, G);
    k_dots<R, M><<<g, kRedThreads, 0, st>>>(psi, Vb, cap, W, na, i0, ks, k, partials);
    return g;
}

template <typename R, int M = 1>
static int launch_update(int m, int G, cudaStream_t st, const void* psi, const void* Vb,
                         size_t cap, typename Cx<R>::T* W, const int64_t* na, int i0,
                         const KrylovScalars* ks, int k, int want_norm, double* partials) {
    if constexpr (M < kMaxM) {
        if (m != M)
            return launch_update<R, M + 1>(m, G, st, psi, Vb, cap, W, na, i0, ks, k, want_norm,
                                           partials);
    }
    static const int g = one_wave_grid(k_update<R, M>, G);
    k_update<R, M><<<g, kRedThreads, 0, st>>>(psi, Vb, cap, W, na, i0, ks, k, want_norm,
                                               partials);
    return g;
}

// beta_k = ||W||; breakdown test; sigma_{k+1} = 1/beta_k.
__global__ void k_update_done(const double* partials, int G, KrylovScalars* ks, int k,
                              int64_t* err) {
    __shared__ double tot[1];
    if (ks->keff <= k) return;
    sum_partials(partials, G, 1, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double b = sqrt(tot[0]);
        if (!isfinite(b)) {
            *err |= 2;
            ks->keff = k + 1;
            return;
        }
        if (b <= 1e-12 * sqrt(ks->hnorm2)) {   // invariant subspace: stop here
            ks->keff = k + 1;
            ks->beta[k] = 0.0;
            return;
        }
        ks->beta[k] = b;
        ks->sigma[k + 1] = 1.0 / b;
    }
}

// ------------------------------------------------ small exponential
// exp(-i T dt) e_1 of the keff x keff Lanczos tridiagonal, one warp, lane r =
// row r.  The spectrum is shifted to its centre (T' = T - mu, the phase
// exp(-i mu dt) applied at the end) and scaled into [-1, 1] by its Gershgorin
// bound g; then exp(-i x R) with R = g |dt| is the Chebyshev series
// J_0(R) + 2 sum_k (-i)^k J_k(R) T_k(x) (Jacobi-Anger), summed with the
// three-term recurrence on the vector.  The Bessel values come from Miller's
// backward recurrence normalised by J_0 + 2 sum J_2k = 1.  R above kChebR is
// split into equal sub-steps, at most kChebSub of them: a larger R (a blown-up
// tridiagonal) sets the numerical-failure bit instead of looping on.  The loop
// body is FMAs and shuffles: FP64 division and square root, slow on this
// part, stay out of it.
// coef_j = beta_0 sigma_j [exp(-i T dt) e_1]_j.
constexpr double kChebR = 2000.0;
constexpr int kChebN = 2304;   // > kChebR + 16 kChebR^(1/3) + 40
constexpr int kChebSub = 64;

// Lane r < n receives [exp(-i T_n dt) e_1]_r for the leading n x n block of
// the Lanczos tridiagonal; false when g |dt| exceeds the sub-step limit.
// Every lane of the warp must call it (shuffles); J: kChebN + 2 shared doubles.
__device__ bool tridiag_exp_lanes(const KrylovScalars* ks, int n, double dt, double* J,
                                  double& out_re, double& out_im) {
    const int r = threadIdx.x & 31;
    const bool on = r < n;
    const double al = on ? ks->alpha[r] : 0.0;
    const double bu0 = (on && r + 1 < n) ? ks->beta[r] : 0.0;            // T[r][r+1]
    const double bup = __shfl_up_sync(0xffffffffu, bu0, 1);   // every lane takes part
    const double bl0 = r > 0 ? bup : 0.0;                        // T[r][r-1]
    double amax = on ? al : -1e300, amin = on ? al : 1e300;
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        amin = fmin(amin, __shfl_xor_sync(0xffffffffu, amin, o));
    }
    const double mu = 0.5 * (amax + amin);
    const double a0 = on ? al - mu : 0.0;
    double g = fabs(a0) + fabs(bl0) + fabs(bu0);
    for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    const double Rtot = g * fabs(dt);
    double vr = r == 0 ? 1.0 : 0.0, vi = 0.0;
    out_re = 0.0;
    out_im = 0.0;
    if (!(Rtot <= kChebR * kChebSub)) return false;   // also NaN
    if (Rtot > 1e-300) {
        const int nsub = (int)ceil(Rtot / kChebR);
        const double R = Rtot / nsub;
        // <= kChebN for R <= kChebR; the clamp only keeps absurd R in bounds
        const int N = (int)fmin(ceil(R + 16.0 * cbrt(R) + 40.0), (double)kChebN);
        // Bessel J_k(R), k = 0..N, unnormalised, by lane 0
        if (r == 0) {
            const double two_over_R = 2.0 / R;
            J[N + 1] = 0.0;
            J[N] = 1e-300;
            for (int k = N; k > 0; --k) {
                const double jm = (k * two_over_R) * J[k] - J[k + 1];
                J[k - 1] = jm;
                if (fabs(jm) > 1e200)
                    for (int q = k - 1; q <= N; ++q) J[q] *= 1e-200;
            }
        }
        __syncwarp();
        double part = 0.0;
        for (int k = 2 + 2 * r; k <= N; k += 64) part += J[k];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const double norm = 1.0 / (J[0] + 2.0 * part);
        const double f = (dt >= 0 ? 1.0 : -1.0) / g;
        const double a = a0 * f, bl = bl0 * f, bu = bu0 * f;
        for (int sub = 0; sub < nsub; ++sub) {
            // p0 = T_0 v, p1 = T_1 v, acc = sum c_k T_k v
            double p0r = vr, p0i = vi;
            double p1r, p1i;
            {
                const double ur = __shfl_up_sync(0xffffffffu, p0r, 1);
                const double ui = __shfl_up_sync(0xffffffffu, p0i, 1);
                const double dr = __shfl_down_sync(0xffffffffu, p0r, 1);
                const double di = __shfl_down_sync(0xffffffffu, p0i, 1);
                p1r = a * p0r + bl * ur + bu * dr;
                p1i = a * p0i + bl * ui + bu * di;
            }
            const double c0 = J[0] * norm, c1 = 2.0 * J[1] * norm;
            double ar = c0 * p0r + c1 * p1i;   // (-i) c1 (p1r + i p1i)
            double ai = c0 * p0i - c1 * p1r;
            for (int k = 2; k <= N; ++k) {
                const double ur = __shfl_up_sync(0xffffffffu, p1r, 1);
                const double ui = __shfl_up_sync(0xffffffffu, p1i, 1);
                const double dr = __shfl_down_sync(0xffffffffu, p1r, 1);
                const double di = __shfl_down_sync(0xffffffffu, p1i, 1);
                const double p2r = 2.0 * (a * p1r + bl * ur + bu * dr) - p0r;
                const double p2i = 2.0 * (a * p1i + bl * ui + bu * di) - p0i;
                const double ck = 2.0 * J[k] * norm;
                switch (k & 3) {   // (-i)^k
                    case 0: ar += ck * p2r; ai += ck * p2i; break;
                    case 1: ar += ck * p2i; ai -= ck * p2r; break;
                    case 2: ar -= ck * p2r; ai -= ck * p2i; break;
                    default: ar -= ck * p2i; ai += ck * p2r; break;
                }
                p0r = p1r; p0i = p1i;
                p1r = p2r; p1i = p2i;
            }
            vr = ar;
            vi = ai;
        }
    }
    double sn, cs;
    sincos(-mu * dt, &sn, &cs);   // exp(-i mu dt)
    out_re = cs * vr - sn * vi;
    out_im = cs * vi + sn * vr;
    return true;
}

__global__ void __launch_bounds__(32) k_tridiag_exp(KrylovScalars* ks, double dt, int64_t* err) {
    __shared__ double J[kChebN + 2];
    const int n = ks->keff;
    const int r = threadIdx.x;
    if (n <= 0) return;
    double vr, vi;
    const bool ok = tridiag_exp_lanes(ks, n, dt, J, vr, vi);
    if (!ok && r == 0) *err |= 2;
    if (r < n) {
        // ks->renorm: the FP32-mix norm correction of the previous step (0 or 1: none)
        const double g = ks->renorm > 0.0 ? ks->renorm : 1.0;
        const double f = ok ? ks->beta0 * ks->sigma[r] * g : 0.0;
        ks->coef[2 * r] = vr * f;
        ks->coef[2 * r + 1] = vi * f;
    }
}

// Error-controlled Krylov order: after Lanczos step k (beta_k known), the
// estimate beta_k |[exp(-i T_{k+1} dt) e_1]_k| of the relative error of the
// order-(k+1) step; at or below tol the step stops at k + 1 vectors.
__global__ void __launch_bounds__(32) k_sil_errcheck(KrylovScalars* ks, int k, double dt,
                                                     double tol) {
    __shared__ double J[kChebN + 2];
    if (ks->keff <= k + 1) return;   // already stopped
    double vr, vi;
    const bool ok = tridiag_exp_lanes(ks, k + 1, dt, J, vr, vi);
    const double ck = __shfl_sync(0xffffffffu, sqrt(vr * vr + vi * vi), k);
    if (threadIdx.x == 0 && ok && ks->beta[k] * ck <= tol) ks->keff = k + 1;
}

// psi <- sum_{j < keff} coef_j V_j  (V_0 is psi itself: read before write).
// partials (nullable): block partials of ||psi||^2 of the result.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_combine(void* psi, const void* Vb, size_t cap,
                                                          const int64_t* na,
                                                          const KrylovScalars* ks, double* partials) {
    using V = typename Cx<R>::T;
    constexpr int kBatch = 4;   // vector loads in flight per thread
    __shared__ R sc[2 * kMaxK];
    const int n_k = ks->keff;
    if (n_k <= 0) return;   // uniform; the norm keeping then ignores the partials
    for (int j = threadIdx.x; j < 2 * n_k; j += blockDim.x) sc[j] = (R)ks->coef[j];
    __syncthreads();
    const int64_t n = min(*na, (int64_t)cap);
    Acc<R> an;
    an.init();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        R ax = 0, ay = 0;
        // j ascending, as a plain loop would sum; the loads of a batch issue
        // before its products
        int j = 0;
        for (; j + kBatch <= n_k; j += kBatch) {
            V v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) v[u] = kvec<R>(psi, Vb, cap, j + u)[p];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const R cr = sc[2 * (j + u)], ci = sc[2 * (j + u) + 1];
                ax += cr * v[u].x - ci * v[u].y;
                ay += cr * v[u].y + ci * v[u].x;
            }
        }
        for (; j < n_k; ++j) {
            const V v = kvec<R>(psi, Vb, cap, j)[p];
            const R cr = sc[2 * j], ci = sc[2 * j + 1];
            ax += cr * v.x - ci * v.y;
            ay += cr * v.y + ci * v.x;
        }
        ((V*)psi)[p] = cmake<R>(ax, ay);
        an.add(ax * ax + ay * ay);
    }
    if (partials) {
        const double vals[1] = {an.value()};
        block_partials<1>(vals, partials);
    }
}

// FP32-mix: norm keeping of the SIL step.  In exact arithmetic the step keeps
// the norm (exp(-i T dt) is unitary and the Krylov basis orthonormal), so the
// norm changes only where the adaption removes coefficients.  With FP32
// coefficients each step's output norm is off by a few 1e-8, which adds up
// over hundreds of steps; a scale that small is below one FP32 unit in the
// last place near 1.  So the run carries in FP64 the norm it should have: the
// target output norm of the step, which follows the adaption (at the next
// step's start, target *= ||psi after prune|| / ||step output||), and the
// factor target / ||step output|| is folded into the next step's
// combination coefficients.  Each output is then off by one step's rounding,
// not by the sum of all of them.
__global__ void k_renorm_factor(const double* partials, int G, KrylovScalars* ks) {
    __shared__ double tot[1];
    sum_partials(partials, G, 1, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double n = sqrt(tot[0]);
        const bool ok = ks->keff > 0 && n > 0.0 && isfinite(n) && ks->rn_target > 0.0;
        ks->renorm = ok ? ks->rn_target / n : 1.0;
        ks->rn_last = ok ? n : 0.0;
    }
}

// ---------------------------------------------------------- observables
// C = sum conj(a0_I) psi_I with a0_I = prod_k f_k(i_k); ||psi||^2; the number
// of active points with |a| < theta.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_observe(const uint32_t* __restrict__ keys,
                                                          const typename Cx<R>::T* __restrict__ psi,
                                                          const int64_t* na, int64_t cap,
                                                          Lattice L, const typename Cx<R>::T* fac,
                                                          double theta2, float lo, float hi,
                                                          double* partials) {
    const int64_t n = min(*na, cap);
    Acc<R> cr, ci, nn;
    cr.init();
    ci.init();
    nn.init();
    double wasted = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = keys[p];
        R ar = 1, ai = 0;
        for (int k = 0; k < L.D; ++k) {
            const int d = (int)((key / L.stride[k]) % (uint32_t)L.n[k]);
            const auto f = fac[k * kMaxN + d];
            const R nr = ar * f.x - ai * f.y;
            const R ni = ar * f.y + ai * f.x;
            ar = nr;
            ai = ni;
        }
        const auto v = psi[p];
        cr.add(ar * v.x + ai * v.y);
        ci.add(ar * v.y - ai * v.x);
        nn.add(v.x * v.x + v.y * v.y);
        bool sig;
        if (sizeof(R) == 8)
            sig = significant64((double)v.x, (double)v.y, theta2);
        else
            sig = significant32((float)v.x, (float)v.y, theta2, lo, hi);
        if (!sig) wasted += 1.0;
    }
    const double vals[4] = {cr.value(), ci.value(), nn.value(), wasted};
    block_partials<4>(vals, partials);
}

// rec = [t, C re, C im, norm2, E (filled later), n_active, n_wasted, keff]
__global__ void k_observe_done(const double* partials, int G, const int64_t* cnt,
                               const KrylovScalars* ks, double t, double* rec) {
    __shared__ double tot[4];
    sum_partials(partials, G, 4, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        rec[0] = t;
        rec[1] = tot[0];
        rec[2] = tot[1];
        rec[3] = tot[2];
        rec[4] = 0.0;
        rec[5] = (double)cnt[CNT_NA];
        rec[6] = tot[3];
        rec[7] = ks ? (double)ks->keff : 0.0;
    }
}

// ------------------------------------------------------------- drivers
static void guard(double theta2, float* lo, float* hi) {
    if (theta2 < 1e-30) {
        *lo = -1.0f;
        *hi = 3.0e38f;
    } else {
        *lo = (float)(theta2 * (1.0 - 1e-5));
        *hi = (float)(theta2 * (1.0 + 1e-5));
    }
}

template <typename R>
static pq_status observe_t(State& s, double theta, double* rec, cudaStream_t st) {
    const int G = red_blocks();
    float lo, hi;
    guard(theta * theta, &lo, &hi);
    const void* fac = sizeof(R) == 8 ? (const void*)s.fac64 : (const void*)s.fac32;
    k_observe<R><<<G, kRedThreads, 0, st>>>(s.keys, (const typename Cx<R>::T*)s.psi,
                                            s.cnt + CNT_NA, (int64_t)s.cap, s.lat,
                                            (const typename Cx<R>::T*)fac, theta * theta, lo, hi,
                                            s.red_tmp);
    PQ_CHECK_LAUNCH();
    k_observe_done<<<1, 256, 0, st>>>(s.red_tmp, G, s.cnt, s.ks, s.t, rec);
    PQ_CHECK_LAUNCH();
    return PQ_OK;
}

static pq_status observe_rec(State& s, double theta, double* rec, cudaStream_t st) {
    return s.prec == PQ_FP64 ? observe_t<double>(s, theta, rec, st)
                             : observe_t<float>(s, theta, rec, st);
}

template <typename R>
static pq_status sil_step(State& s, const pq_prop_desc& d, double* prev_E, cudaStream_t st) {
    using V = typename Cx<R>::T;
    const int G = red_blocks();
    const size_t cap = s.cap;
    const int K = d.K;
    k_norm2<R><<<G, kRedThreads, 0, st>>>((const V*)s.psi, s.cnt + CNT_NA, (int64_t)cap, s.red_tmp);
    PQ_CHECK_LAUNCH();
    k_start_step<<<1, 256, 0, st>>>(s.red_tmp, G, s.ks, K, s.cnt + CNT_ERR, sizeof(R) == 4 ? 1 : 0);
    PQ_CHECK_LAUNCH();
    pq_status rc;
    for (int k = 0; k < K; ++k) {
        const void* in = k == 0 ? s.psi : (const void*)((V*)s.V + (size_t)(k - 1) * cap);
        V* W = (V*)s.V + (size_t)k * cap;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (s.timing.enabled) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, st);
        }
        rc = apply_H_launch(s, in, W, s.prec, &s.ks->sigma[k], &s.ks->keff, k, st);
        if (rc) return rc;
        if (s.timing.enabled) {
            cudaEventRecord(e1, st);
            s.timing.ev_start.push_back(e0);
            s.timing.ev_stop.push_back(e1);
        }
        // which previous vectors to orthogonalise against
        int i0 = 0;
        if (k == K - 1) i0 = k;                   // only alpha_k needed
        else if (!d.reorth) i0 = k > 0 ? k - 1 : 0;
        for (int c0 = i0; c0 <= k; c0 += kMaxM) {
            const int m = min(kMaxM, k - c0 + 1);
            const int g = launch_dots<R>(m, G, st, s.psi, s.V, cap, W, s.cnt + CNT_NA, c0, s.ks,
                                         k, s.red_tmp);
            PQ_CHECK_LAUNCH();
            k_dots_done<<<1, 256, 0, st>>>(s.red_tmp, g, c0, m, s.ks, k, prev_E, s.cnt + CNT_ERR);
            PQ_CHECK_LAUNCH();
        }
        if (k == K - 1) break;
        int g_norm = G;   // blocks of the update that summed ||W||^2
        for (int c0 = i0; c0 <= k; c0 += kMaxM) {
            const int m = min(kMaxM, k - c0 + 1);
            const bool last = c0 + m > k;
            g_norm = launch_update<R>(m, G, st, s.psi, s.V, cap, W, s.cnt + CNT_NA, c0, s.ks, k,
                                      last ? 1 : 0, s.red_tmp);
            PQ_CHECK_LAUNCH();
        }
        k_update_done<<<1, 256, 0, st>>>(s.red_tmp, g_norm, s.ks, k, s.cnt + CNT_ERR);
        PQ_CHECK_LAUNCH();
        if (d.sil_tol > 0.0) {
            k_sil_errcheck<<<1, 32, 0, st>>>(s.ks, k, d.dt, d.sil_tol);
            PQ_CHECK_LAUNCH();
        }
    }
    k_tridiag_exp<<<1, 32, 0, st>>>(s.ks, d.dt, s.cnt + CNT_ERR);
    PQ_CHECK_LAUNCH();
    // FP32-mix: the combination also sums the output's norm for the next step's
    // norm correction
    static const int g_comb = one_wave_grid(k_combine<R>, G);
    k_combine<R><<<g_comb, kRedThreads, 0, st>>>(s.psi, s.V, cap, s.cnt + CNT_NA, s.ks,
                                                 sizeof(R) == 4 ? s.red_tmp : nullptr);
    PQ_CHECK_LAUNCH();
    if (sizeof(R) == 4) {
        k_renorm_factor<<<1, 256, 0, st>>>(s.red_tmp, g_comb, s.ks);
        PQ_CHECK_LAUNCH();
    }
    return PQ_OK;
}

// ------------------------------------------------------------------ RK4
// Classical fourth-order Runge-Kutta step of i da/dt = H a (an alternative to
// SIL; not in the paper): k_s = -i H y_s with y_1 = a, y_2 = a + dt/2 k_1,
// y_3 = a + dt/2 k_2, y_4 = a + dt k_3; a' = a + dt/6 (k_1 + 2 k_2 + 2 k_3 + k_4).
// Buffers: Krylov slots 0 (next stage input), 1 (H y), 2 (accumulated a').
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_rk4_energy(const typename Cx<R>::T* __restrict__ a,
                                                             const typename Cx<R>::T* __restrict__ Ha,
                                                             const int64_t* na, int64_t cap,
                                                             double* partials) {
    const int64_t n = min(*na, cap);
    Acc<R> e, nn;
    e.init();
    nn.init();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const auto x = a[p], y = Ha[p];
        e.add(x.x * y.x + x.y * y.y);
        nn.add(x.x * x.x + x.y * x.y);
    }
    const double vals[2] = {e.value(), nn.value()};
    block_partials<2>(vals, partials);
}

__global__ void k_rk4_energy_done(const double* partials, int G, double* E) {
    __shared__ double tot[2];
    sum_partials(partials, G, 2, tot);
    __syncthreads();
    if (threadIdx.x == 0 && E) *E = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
}

// stage 0: acc = a + c_acc t, next = a + c_next t;  stages 1, 2: acc += c_acc t,
// next = a + c_next t;  stage 3: a = acc + c_acc t;  t = -i H y.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_rk4_stage(typename Cx<R>::T* a,
                                                            const typename Cx<R>::T* __restrict__ Hy,
                                                            typename Cx<R>::T* next,
                                                            typename Cx<R>::T* acc, const int64_t* na,
                                                            int64_t cap, R c_acc, R c_next,
                                                            int stage) {
    using V = typename Cx<R>::T;
    const int64_t n = min(*na, cap);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const V h = Hy[p];
        const V t = cmake<R>(h.y, -h.x);   // -i (h.x + i h.y)
        if (stage == 3) {
            const V c = acc[p];
            a[p] = cmake<R>(c.x + c_acc * t.x, c.y + c_acc * t.y);
            continue;
        }
        const V x = a[p];
        V c = stage == 0 ? x : acc[p];
        c.x += c_acc * t.x;
        c.y += c_acc * t.y;
        acc[p] = c;
        next[p] = cmake<R>(x.x + c_next * t.x, x.y + c_next * t.y);
    }
}

template <typename R>
static pq_status rk4_step(State& s, const pq_prop_desc& d, double* prev_E, cudaStream_t st) {
    using V = typename Cx<R>::T;
    const int G = red_blocks();
    const size_t cap = s.cap;
    V* next = (V*)s.V;
    V* Hy = (V*)s.V + cap;
    V* acc = (V*)s.V + 2 * cap;
    const R dt = (R)d.dt;
    const R c_acc[4] = {dt / 6, dt / 3, dt / 3, dt / 6};
    const R c_next[4] = {dt / 2, dt / 2, dt, 0};
    for (int stage = 0; stage < 4; ++stage) {
        const void* in = stage == 0 ? s.psi : (const void*)next;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (s.timing.enabled) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, st);
        }
        pq_status rc = apply_H_launch(s, in, Hy, s.prec, nullptr, nullptr, 0, st);
        if (rc) return rc;
        if (s.timing.enabled) {
            cudaEventRecord(e1, st);
            s.timing.ev_start.push_back(e0);
            s.timing.ev_stop.push_back(e1);
        }
        if (stage == 0) {   // E of the state at the start of the step
            k_rk4_energy<R><<<G, kRedThreads, 0, st>>>((const V*)s.psi, Hy, s.cnt + CNT_NA,
                                                       (int64_t)cap, s.red_tmp);
            PQ_CHECK_LAUNCH();
            k_rk4_energy_done<<<1, 256, 0, st>>>(s.red_tmp, G, prev_E);
            PQ_CHECK_LAUNCH();
        }
        k_rk4_stage<R><<<G, kRedThreads, 0, st>>>((V*)s.psi, Hy, next, acc, s.cnt + CNT_NA,
                                                  (int64_t)cap, c_acc[stage], c_next[stage], stage);
        PQ_CHECK_LAUNCH();
    }
    return PQ_OK;
}

pq_status ensure_krylov(State& s, int K) {
    if (s.V_K >= K) return PQ_OK;
    if (s.V) {
        cudaDeviceSynchronize();   // the old space may still be in use on some stream
        dev_free(s.V, 0, false);
    }
    s.V = nullptr;
    s.V_K = 0;
    s.V = dev_alloc((size_t)K * s.cap * s.esize, 0, false);
    if (!s.V) {
        cudaGetLastError();
        set_error("cannot allocate the Krylov space (%zu bytes)", (size_t)K * s.cap * s.esize);
        return PQ_ENOMEM;
    }
    s.V_K = K;
    return PQ_OK;
}

pq_status sil_only(State& s, const pq_prop_desc& d, cudaStream_t st) {
    pq_status rc = ensure_krylov(s, d.K);
    if (rc) return rc;
    return s.prec == PQ_FP64 ? sil_step<double>(s, d, nullptr, st) : sil_step<float>(s, d, nullptr, st);
}

pq_status propagate_impl(State& s, const pq_prop_desc& d, int nsteps, cudaStream_t st) {
    if (d.K < 1 || d.K > kMaxK) {
        set_error("Krylov dimension %d outside 1..%d", d.K, kMaxK);
        return PQ_EINVAL;
    }
    if (!(d.dt > 0) || !(d.theta >= 0) || nsteps < 0) {
        set_error("need dt > 0, theta >= 0, nsteps >= 0");
        return PQ_EINVAL;
    }
    if (d.integrator != PQ_SIL && d.integrator != PQ_RK4) {
        set_error("unknown integrator %d (0: SIL, 1: RK4)", d.integrator);
        return PQ_EINVAL;
    }
    const bool rk4 = d.integrator == PQ_RK4;
    if (!(d.sil_tol >= 0) || !std::isfinite(d.sil_tol)) {
        set_error("sil_tol must be finite and >= 0");
        return PQ_EINVAL;
    }
    pq_status erc = check_neighbour_rule(s.lat, d.radius);
    if (erc) return erc;
    erc = ensure_krylov(s, rk4 ? std::max(d.K, 3) : d.K);
    if (erc) return erc;
    if (nsteps == 0) return PQ_OK;
    // FP32 H.psi path hint: the set size now, then the size after step n - 2
    // read back without blocking (two pinned slots and events).  The hint only
    // picks between two correct paths, so without the events it stays as set.
    cudaEvent_t hev[2] = {nullptr, nullptr};
    bool hinted = s.prec != PQ_FP64;
    if (hinted) {
        if (!s.h_na && cudaMallocHost((void**)&s.h_na, 2 * sizeof(int64_t)) != cudaSuccess) {
            s.h_na = nullptr;
            set_error("cudaMallocHost failed");
            return PQ_ENOMEM;
        }
        PQ_CUDA_TRY(cudaMemcpyAsync(s.h_na, s.cnt + CNT_NA, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PQ_CUDA_TRY(cudaStreamSynchronize(st));
        s.dense_hint = 2 * s.h_na[0] >= (int64_t)s.lat.nfull ? 1 : 0;
        if (cudaEventCreateWithFlags(&hev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&hev[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (cudaEvent_t& e : hev)
                if (e) cudaEventDestroy(e), e = nullptr;
            hinted = false;
        }
    }
    double* recs = nullptr;
    recs = (double*)dev_alloc((size_t)(nsteps + 1) * 8 * sizeof(double), st, true);
    if (!recs) {
        for (cudaEvent_t e : hev)
            if (e) cudaEventDestroy(e);
        set_error("device allocation of the step records failed");
        return PQ_ENOMEM;
    }
    if (cudaMemsetAsync(recs, 0, (size_t)(nsteps + 1) * 8 * sizeof(double), st) != cudaSuccess) {
        for (cudaEvent_t e : hev)
            if (e) cudaEventDestroy(e);
        dev_free(recs, st, true);
        set_error("clearing the step records failed");
        return PQ_ECUDA;
    }
    // Slot 0 receives E of the record already on the host (alpha_0 of step 1).
    pq_status rc = PQ_OK;
    for (int n = 0; n < nsteps && rc == PQ_OK; ++n) {
        if (hinted && n >= 2 && cudaEventQuery(hev[n & 1]) == cudaSuccess)
            s.dense_hint = 2 * s.h_na[n & 1] >= (int64_t)s.lat.nfull ? 1 : 0;
        double* prevE = recs + (size_t)n * 8 + 4;
        if (rk4)
            rc = s.prec == PQ_FP64 ? rk4_step<double>(s, d, prevE, st) : rk4_step<float>(s, d, prevE, st);
        else
            rc = s.prec == PQ_FP64 ? sil_step<double>(s, d, prevE, st) : sil_step<float>(s, d, prevE, st);
        if (rc) break;
        rc = prune_launch(s, d.theta, d.radius, d.rel_excl, st);
        if (rc) break;
        if (hinted) {
            cudaMemcpyAsync(s.h_na + (n & 1), s.cnt + CNT_NA, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
            cudaEventRecord(hev[n & 1], st);
        }
        s.t += d.dt;
        rc = observe_rec(s, d.theta, recs + (size_t)(n + 1) * 8, st);
    }
    std::vector<double> h((size_t)(nsteps + 1) * 8);
    cudaError_t e1 = cudaMemcpyAsync(h.data(), recs, h.size() * sizeof(double),
                                     cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaMemcpyAsync(s.h_cnt, s.cnt, CNT_SIZE * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st);
    cudaError_t e3 = cudaStreamSynchronize(st);
    dev_free(recs, st, true);
    for (cudaEvent_t e : hev)
        if (e) cudaEventDestroy(e);
    if (hinted && e3 == cudaSuccess) s.dense_hint = 2 * s.h_cnt[CNT_NA] >= (int64_t)s.lat.nfull ? 1 : 0;
    if (rc) return rc;
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        set_error("propagate: %s", cudaGetErrorString(e3 != cudaSuccess ? e3 : (e1 ? e1 : e2)));
        return PQ_ECUDA;
    }
    // E of the previous newest host record
    if (!s.obs.empty() && s.obs_energy_pending) {
        s.obs.back().energy = h[4];
        s.obs_energy_pending = false;
    }
    for (int n = 1; n <= nsteps; ++n) {
        const double* r = &h[(size_t)n * 8];
        // E of record n is alpha_0 of step n+1, stored in slot n
        ObsRecord o{r[0], r[1], r[2], r[3], n < nsteps ? r[4] : 0.0, (int64_t)r[5],
                    (int64_t)r[6]};
        s.obs.push_back(o);
    }
    s.obs_energy_pending = true;
    if (s.timing.enabled) {
        for (size_t i = 0; i < s.timing.ev_start.size(); ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, s.timing.ev_start[i], s.timing.ev_stop[i]);
            s.timing.ms += ms;
            cudaEventDestroy(s.timing.ev_start[i]);
            cudaEventDestroy(s.timing.ev_stop[i]);
        }
        s.timing.n_apply += (int64_t)s.timing.ev_start.size();
        // active points per H.psi: the set before each step (record n-1)
        const size_t base = s.obs.size() - nsteps;
        for (int n = 0; n < nsteps; ++n) {
            const double na_before = (double)s.obs[base + n - 1].n_active;
            s.timing.coef += na_before * (rk4 ? 4 : d.K);
        }
        s.timing.ev_start.clear();
        s.timing.ev_stop.clear();
    }
    if (s.h_cnt[CNT_FAULT]) {
        set_error("bounds check failed: site %lld, index %lld, bound %lld",
                  (long long)s.h_cnt[CNT_FAULT], (long long)s.h_cnt[CNT_FAULT + 1],
                  (long long)s.h_cnt[CNT_FAULT + 2]);
        return PQ_EINVAL;
    }
    const int64_t errw = s.h_cnt[CNT_ERR];
    if (errw & 1) {
        set_error("active set outgrew the capacity (%lld > %zu)", (long long)s.h_cnt[CNT_NA], s.cap);
        return PQ_ECAPACITY;
    }
    if (errw & 2) {
        set_error("non-finite norm or Lanczos coefficient");
        return PQ_ENUMERIC;
    }
    return PQ_OK;
}

pq_status observe_launch(State& s, double theta, cudaStream_t st) {
    double* rec = nullptr;
    rec = (double*)dev_alloc(8 * sizeof(double), st, true);
    if (!rec) {
        set_error("device allocation failed");
        return PQ_ENOMEM;
    }
    pq_status rc = observe_rec(s, theta, rec, st);
    double h[8] = {0};
    cudaMemcpyAsync(h, rec, sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    dev_free(rec, st, true);
    if (rc) return rc;
    if (e != cudaSuccess) {
        set_error("observe: %s", cudaGetErrorString(e));
        return PQ_ECUDA;
    }
    s.obs.push_back(ObsRecord{h[0], h[1], h[2], h[3], 0.0, (int64_t)h[5], (int64_t)h[6]});
    s.obs_energy_pending = true;
    return PQ_OK;
}

// E = Re<psi|H psi> / ||psi||^2 of the current state (one extra H.psi).
template <typename R>
static pq_status energy_t(State& s, double* E, cudaStream_t st) {
    using V = typename Cx<R>::T;
    const int G = red_blocks();
    void* W = nullptr;
    W = dev_alloc(s.cap * s.esize, st, true);
    if (!W) {
        set_error("device allocation failed");
        return PQ_ENOMEM;
    }
    k_norm2<R><<<G, kRedThreads, 0, st>>>((const V*)s.psi, s.cnt + CNT_NA, (int64_t)s.cap, s.red_tmp);
    PQ_CHECK_LAUNCH();
    k_start_step<<<1, 256, 0, st>>>(s.red_tmp, G, s.ks, 1, s.cnt + CNT_ERR);
    PQ_CHECK_LAUNCH();
    // W = H (psi / ||psi||); <psi/||psi||, W> is then E
    pq_status rc = apply_H_launch(s, s.psi, W, s.prec, &s.ks->sigma[0], nullptr, 0, st);
    if (rc) {
        dev_free(W, st, true);
        return rc;
    }
    k_dots<R, 1><<<G, kRedThreads, 0, st>>>(s.psi, s.V, s.cap, (const V*)W, s.cnt + CNT_NA, 0,
                                            s.ks, 0, s.red_tmp);
    PQ_CHECK_LAUNCH();
    double* dE = nullptr;
    dE = (double*)dev_alloc(sizeof(double), st, true);
    if (!dE) {
        dev_free(W, st, true);
        set_error("device allocation failed");
        return PQ_ENOMEM;
    }
    PQ_CUDA_TRY(cudaMemsetAsync(dE, 0, sizeof(double), st));
    k_dots_done<<<1, 256, 0, st>>>(s.red_tmp, G, 0, 1, s.ks, 0, dE, s.cnt + CNT_ERR);
    PQ_CHECK_LAUNCH();
    double h = 0.0;
    cudaMemcpyAsync(&h, dE, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    dev_free(dE, st, true);
    dev_free(W, st, true);
    if (e != cudaSuccess) {
        set_error("energy: %s", cudaGetErrorString(e));
        return PQ_ECUDA;
    }
    *E = h;
    return PQ_OK;
}

pq_status energy_of_current(State& s, double* E, cudaStream_t st) {
    return s.prec == PQ_FP64 ? energy_t<double>(s, E, st) : energy_t<float>(s, E, st);
}

}  // namespace pq
