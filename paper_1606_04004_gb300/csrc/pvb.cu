// Pruned dynamics in the biorthogonal projected von Neumann basis (Sec. 2.2).
//
// The basis is nonorthogonal (i S da/dt = H a, H = B^dagger H^chi B,
// S = B^dagger B, Eq. pvb_H_trafo).  Because partially transformed tensors are
// not sparse in this basis (Sec. 2.2.2, drawbacks in high dimensions), H_AA a
// is formed on the full grid,
//     y = P_A (x_k B_k^dagger) H^chi (x_k B_k) P_A^T a,
// and S_AA^{-1} y by conjugate gradients with S_AA v = P_A (x_k S_k) P_A^T v.
// Propagation: Lanczos in the S inner product <x, y>_S = x^dagger S_AA y, for
// which S_AA^{-1} H_AA is self-adjoint; FP64 scalars on the host (each Krylov
// vector needs a CG solve, so the step is host-orchestrated).
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "device_util.cuh"

namespace pq {

constexpr int kPvbThreads = 256;
using cd = std::complex<double>;

// X[g] = a[rank(g)] for active lattice points g, 0 elsewhere: the whole grid
// in one pass (the active set's bitmap and rank offsets give the position).
// `gate` (nullable): nothing to do while *gate != 0 (a converged solve).
template <typename R>
__global__ void k_embed_full(const uint64_t* __restrict__ bits, const uint32_t* __restrict__ off,
                             const typename Cx<R>::T* __restrict__ a, uint32_t nfull,
                             typename Cx<R>::T* __restrict__ X, const double* gate) {
    if (gate && *gate != 0.0) return;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nfull; g += gridDim.x * blockDim.x)
        X[g] = bit_test(bits, g) ? a[rank_of(bits, off, g)] : cmake<R>(0, 0);
}

// y[p] = Y[key[p]]
template <typename R>
__global__ void k_restrict(const uint32_t* __restrict__ keys, const typename Cx<R>::T* __restrict__ Y,
                           const int64_t* na, int64_t cap, typename Cx<R>::T* __restrict__ y,
                           const double* gate) {
    if (gate && *gate != 0.0) return;
    const int64_t n = min(*na, cap);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        y[p] = Y[keys[p]];
}

// Full-grid transform along mode k with a complex n x n matrix M (row
// stride kMaxN, interleaved): Y[o, i, in] (+)= sum_j M[i][j] X[o, j, in].
// Threads: inner index fastest when the mode has an inner extent, else the
// output index i fastest (M read transposed from shared memory).
template <typename R>
__global__ void __launch_bounds__(kPvbThreads) k_grid_mode(
    const typename Cx<R>::T* __restrict__ X, typename Cx<R>::T* __restrict__ Y,
    const R* __restrict__ M, int nk, uint32_t inner, uint32_t total, int accumulate,
    const double* gate) {
    using V = typename Cx<R>::T;
    if (gate && *gate != 0.0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    V* Ms = reinterpret_cast<V*>(smem);   // Ms[j * nk + i] = M[i][j]
    for (int e = threadIdx.x; e < nk * nk; e += blockDim.x) {
        const int i = e % nk, j = e / nk;
        Ms[e] = cmake<R>(M[((size_t)i * kMaxN + j) * 2], M[((size_t)i * kMaxN + j) * 2 + 1]);
    }
    __syncthreads();
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        uint32_t o, i, in;
        if (inner > 1) {
            in = t % inner;
            const uint32_t q = t / inner;
            i = q % nk;
            o = q / nk;
        } else {
            in = 0;
            i = t % nk;
            o = t / nk;
        }
        const size_t base = (size_t)o * nk * inner + in;
        R ar = 0, ai = 0;
        for (int j = 0; j < nk; ++j) {
            const V m = Ms[j * nk + i];
            const V x = X[base + (size_t)j * inner];
            ar += m.x * x.x - m.y * x.y;
            ai += m.x * x.y + m.y * x.x;
        }
        const size_t oi = base + (size_t)i * inner;
        if (accumulate) {
            const V y = Y[oi];
            ar += y.x;
            ai += y.y;
        }
        Y[oi] = cmake<R>(ar, ai);
    }
}

// The same transform for modes longer than 64 (the matrix stays in global
// memory, read through the cache): the double well's 165- and 81-point grids.
template <typename R>
__global__ void __launch_bounds__(kPvbThreads) k_grid_mode_long(
    const typename Cx<R>::T* __restrict__ X, typename Cx<R>::T* __restrict__ Y,
    const R* __restrict__ M, int nk, uint32_t inner, uint32_t total, int accumulate,
    const double* gate) {
    using V = typename Cx<R>::T;
    if (gate && *gate != 0.0) return;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const uint32_t in = t % inner, q = t / inner;
        const uint32_t i = q % (uint32_t)nk, o = q / (uint32_t)nk;
        const size_t base = (size_t)o * nk * inner + in;
        const R* mrow = M + (size_t)i * kMaxN * 2;
        R ar = 0, ai = 0;
        for (int j = 0; j < nk; ++j) {
            const R mr = mrow[2 * j], mi = mrow[2 * j + 1];
            const V x = X[base + (size_t)j * inner];
            ar += mr * x.x - mi * x.y;
            ai += mr * x.y + mi * x.x;
        }
        const size_t oi = base + (size_t)i * inner;
        if (accumulate) {
            const V y = Y[oi];
            ar += y.x;
            ai += y.y;
        }
        Y[oi] = cmake<R>(ar, ai);
    }
}

// Y = V(x) X on the full grid, V from the SoP potential tables.
template <typename R>
__global__ void k_grid_potential(const typename Cx<R>::T* __restrict__ X,
                                 typename Cx<R>::T* __restrict__ Y, Lattice L,
                                 const R* __restrict__ pot, const R* __restrict__ potc, int nt) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < L.nfull; g += gridDim.x * blockDim.x) {
        R v = 0;
        for (int t = 0; t < nt; ++t) {
            R f = potc[t];
            for (int k = 0; k < L.D; ++k) {
                const int d = (int)((g / L.stride[k]) % (uint32_t)L.n[k]);
                f *= pot[((size_t)t * L.D + k) * kMaxN + d];
            }
            v += f;
        }
        const auto x = X[g];
        Y[g] = cmake<R>(v * x.x, v * x.y);
    }
}

// partials[b] = (re, im) of sum conj(x) y over the block's elements
template <typename R>
__global__ void __launch_bounds__(kPvbThreads) k_cdot(const typename Cx<R>::T* __restrict__ x,
                                                       const typename Cx<R>::T* __restrict__ y,
                                                       int64_t n, double* partials,
                                                       const double* gate = nullptr) {
    if (gate && *gate != 0.0) return;
    double re = 0.0, im = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const auto a = x[p];
        const auto b = y[p];
        re += (double)a.x * b.x + (double)a.y * b.y;
        im += (double)a.x * b.y - (double)a.y * b.x;
    }
    __shared__ double sh[2][kPvbThreads / 32];
    re = warp_sum(re);
    im = warp_sum(im);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = re;
        sh[1][threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int w = 0; w < kPvbThreads / 32; ++w) s += sh[threadIdx.x][w];
        partials[blockIdx.x * 2 + threadIdx.x] = s;
    }
}

// out = a1 x1 + a2 x2 (x2 may be null)
template <typename R>
__global__ void k_lincomb(typename Cx<R>::T* out, double a1r, double a1i,
                          const typename Cx<R>::T* x1, double a2r, double a2i,
                          const typename Cx<R>::T* x2, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const auto u = x1[p];
        double r = a1r * u.x - a1i * u.y, i = a1r * u.y + a1i * u.x;
        if (x2) {
            const auto v = x2[p];
            r += a2r * v.x - a2i * v.y;
            i += a2r * v.y + a2i * v.x;
        }
        out[p] = cmake<R>((R)r, (R)i);
    }
}

// Conjugate-gradient scalars on the device (slots of a small double array),
// so that an iteration needs no host round trip.  Preconditioned CG for
// S_AA x = y with M = P_A (x_k S_k^-1) P_A^T:
//   r = y, z = M r, p = z;  per iteration  alpha = <r,z> / <p,Sp>,
//   x += alpha p, r -= alpha Sp, converged when <r,r> <= tol^2 <y,y>,
//   z = M r, beta = <r,z>_new / <r,z>, p = z + beta p.
enum { kCgRR = 0, kCgY2, kCgAlpha, kCgBeta, kCgDone, kCgFail, kCgIt, kCgRZ, kCgSlots };

// Sum of the real parts of partials[G][2] (fixed order), then the update of
// `mode`: 0 = start (<y,y>: rr and the reference), 3 = start (<r,z>),
// 1 = after <p,Sp> (alpha), 2 = after <r,r> (iteration count, convergence),
// 4 = after the new <r,z> (beta).
__global__ void k_cg_scalar(const double* partials, int G, double* cg, int mode, double tol2) {
    const int lane = threadIdx.x;
    if (mode != 0 && mode != 3 && cg[kCgDone] != 0.0) return;
    double acc = 0.0;
    for (int b = lane; b < G; b += 32) acc += partials[2 * b];
    acc = warp_sum(acc);
    if (lane != 0) return;
    if (mode == 0) {
        cg[kCgRR] = acc;
        cg[kCgY2] = fmax(acc, 1e-300);
        cg[kCgDone] = acc <= tol2 * cg[kCgY2] ? 1.0 : 0.0;
        cg[kCgFail] = 0.0;
        cg[kCgIt] = 0.0;
        return;
    }
    if (mode == 3) {
        cg[kCgRZ] = acc;
        return;
    }
    if (mode == 1) {
        const double al = cg[kCgRZ] / acc;
        if (!isfinite(al)) {
            cg[kCgFail] = 1.0;
            cg[kCgDone] = 1.0;
            return;
        }
        cg[kCgAlpha] = al;
    } else if (mode == 2) {
        cg[kCgRR] = acc;
        cg[kCgIt] += 1.0;
        if (acc <= tol2 * cg[kCgY2]) cg[kCgDone] = 1.0;
    } else {
        cg[kCgBeta] = acc / cg[kCgRZ];
        cg[kCgRZ] = acc;
    }
}

// out = x1 + sign * cg[slot] * x2 (real coefficient), nothing once CG is done.
template <typename R>
__global__ void k_cg_axpy(typename Cx<R>::T* out, const typename Cx<R>::T* x1,
                          const typename Cx<R>::T* x2, int64_t n, const double* cg, int slot,
                          double sign) {
    if (cg[kCgDone] != 0.0) return;
    const double c = sign * cg[slot];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const auto u = x1[p];
        const auto v = x2[p];
        out[p] = cmake<R>((R)(u.x + c * v.x), (R)(u.y + c * v.y));
    }
}

template <typename R>
__global__ void k_packet_bra(const uint32_t* __restrict__ keys, const int64_t* na, int64_t cap,
                             Lattice L, const double2* __restrict__ fac, typename Cx<R>::T* out) {
    const int64_t n = min(*na, cap);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = keys[p];
        double re = 1.0, im = 0.0;
        for (int k = 0; k < L.D; ++k) {
            const int d = (int)((key / L.stride[k]) % (uint32_t)L.n[k]);
            const double2 f = fac[k * kMaxN + d];
            const double nr = re * f.x - im * f.y, ni = re * f.y + im * f.x;
            re = nr;
            im = ni;
        }
        out[p] = cmake<R>((R)re, (R)im);
    }
}

namespace {

template <typename R>
struct Pvb {
    using V = typename Cx<R>::T;
    State& s;
    cudaStream_t st;
    int64_t n;        // active points (host copy)
    V* X;             // full-grid buffers
    V* Y;
    V* Z;
    double* part;
    int G;
    const double* gate = nullptr;   // set during a solve: its kernels stop once it converged

    Pvb(State& s_, cudaStream_t st_) : s(s_), st(st_), n(0) {
        X = (V*)s.pvb_grid;
        Y = X + s.lat.nfull;
        Z = Y + s.lat.nfull;
        part = s.red_tmp;
        G = grid_size() * 2;
    }
    const R* mat(double* m64, float* m32, int k) const {
        return (sizeof(R) == 8 ? (const R*)m64 : (const R*)m32) + (size_t)k * kMaxN * kMaxN * 2;
    }
    pq_status count() {
        PQ_CUDA_TRY(cudaMemcpyAsync(s.h_cnt, s.cnt, CNT_SIZE * 8, cudaMemcpyDeviceToHost, st));
        PQ_CUDA_TRY(cudaStreamSynchronize(st));
        if (s.h_cnt[CNT_ERR] & 1) {
            set_error("active set outgrew the capacity");
            return PQ_ECAPACITY;
        }
        n = std::min<int64_t>(s.h_cnt[CNT_NA], (int64_t)s.cap);
        return PQ_OK;
    }
    // Y (+)= M_k along mode k of X, every mode of the full grid; `real`: M is
    // real (its imaginary parts are zero: the kinetic matrix)
    pq_status mode(const V* in, V* out, const R* M, int k, int acc, bool real = false) {
        const Lattice& L = s.lat;
        const int nk = L.n[k];
        const uint32_t inner = L.stride[k];
        if (sizeof(R) == 4 && nk <= kTcMaxN)   // FP32: tensor cores, split TF32
            return tc_grid_mode(s, (const float2*)in, (float2*)out, (const float*)M, k, acc, real, st,
                                gate);
        if (nk > kMaxNTile) {
            k_grid_mode_long<R><<<grid_size() * 8, kPvbThreads, 0, st>>>(in, out, M, nk, inner,
                                                                         L.nfull, acc, gate);
            PQ_CHECK_LAUNCH();
            return PQ_OK;
        }
        const size_t sm = (size_t)nk * nk * sizeof(V);
        static bool attr = false;
        if (!attr) {
            PQ_CUDA_TRY(cudaFuncSetAttribute(k_grid_mode<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024));
            attr = true;
        }
        k_grid_mode<R><<<grid_size() * 8, kPvbThreads, sm, st>>>(in, out, M, nk, inner, L.nfull, acc,
                                                                 gate);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    }
    // transform by the per-mode matrices (mats selects B, B^dagger or S)
    pq_status all_modes(V*& cur, V*& tmp, double* m64, float* m32) {
        for (int k = 0; k < s.lat.D; ++k) {
            pq_status rc = mode(cur, tmp, mat(m64, m32, k), k, 0);
            if (rc) return rc;
            std::swap(cur, tmp);
        }
        return PQ_OK;
    }
    pq_status embed(const void* a) {
        k_embed_full<R><<<grid_size() * 4, kPvbThreads, 0, st>>>(s.bits, s.off, (const V*)a,
                                                                s.lat.nfull, X, gate);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    }
    pq_status restrict_to(const V* full, void* y) {
        k_restrict<R><<<G, kPvbThreads, 0, st>>>(s.keys, full, s.cnt + CNT_NA, (int64_t)s.cap, (V*)y,
                                                 gate);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    }
    // y = M v = P_A (x_k S_k^-1) P_A^T v, the preconditioner of the S_AA solve
    pq_status Minv(const void* v, void* y) {
        pq_status rc;
        if ((rc = embed(v))) return rc;
        V* cur = X;
        V* tmp = Y;
        if ((rc = all_modes(cur, tmp, s.pvbSi64, s.pvbSi32))) return rc;
        return restrict_to(cur, y);
    }
    // y = H_AA a
    pq_status H(const void* a, void* y) {
        pq_status rc;
        if ((rc = embed(a))) return rc;
        V* cur = X;
        V* tmp = Y;
        if ((rc = all_modes(cur, tmp, s.pvbB64, s.pvbB32))) return rc;   // (x B) a: grid values
        // Z = H^chi cur: potential, then kinetic along every mode
        const R* pot = sizeof(R) == 8 ? (const R*)s.pot64 : (const R*)s.pot32;
        const R* potc = pot + (size_t)std::max(s.nterms, 1) * s.lat.D * kMaxN;
        k_grid_potential<R><<<grid_size() * 8, kPvbThreads, 0, st>>>(cur, Z, s.lat, pot, potc, s.nterms);
        PQ_CHECK_LAUNCH();
        for (int k = 0; k < s.lat.D; ++k)
            if ((rc = mode(cur, Z, mat(s.pvbT64, s.pvbT32, k), k, 1, true))) return rc;
        V* c2 = Z;
        V* t2 = cur;
        if ((rc = all_modes(c2, t2, s.pvbBh64, s.pvbBh32))) return rc;     // (x B^dagger)
        return restrict_to(c2, y);
    }
    // y = S_AA v
    pq_status S(const void* v, void* y) {
        pq_status rc;
        if ((rc = embed(v))) return rc;
        V* cur = X;
        V* tmp = Y;
        if ((rc = all_modes(cur, tmp, s.pvbS64, s.pvbS32))) return rc;
        return restrict_to(cur, y);
    }
    pq_status dot(const void* x, const void* y, cd* out) {
        k_cdot<R><<<G, kPvbThreads, 0, st>>>((const V*)x, (const V*)y, n, part);
        PQ_CHECK_LAUNCH();
        std::vector<double> h((size_t)G * 2);
        PQ_CUDA_TRY(cudaMemcpyAsync(h.data(), part, h.size() * 8, cudaMemcpyDeviceToHost, st));
        PQ_CUDA_TRY(cudaStreamSynchronize(st));
        double re = 0.0, im = 0.0;
        for (int b = 0; b < G; ++b) {
            re += h[2 * b];
            im += h[2 * b + 1];
        }
        *out = cd(re, im);
        return PQ_OK;
    }
    pq_status lin(void* out, cd a1, const void* x1, cd a2 = 0.0, const void* x2 = nullptr) {
        k_lincomb<R><<<G, kPvbThreads, 0, st>>>((V*)out, a1.real(), a1.imag(), (const V*)x1, a2.real(),
                                                a2.imag(), (const V*)x2, n);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    }
    void* vec(int i) { return (char*)s.pvb_vec + (size_t)i * s.cap * sizeof(V); }
    // x = S_AA^{-1} y by preconditioned conjugate gradients (x, y distinct),
    // M = P_A (x_k S_k^-1) P_A^T.  The scalars live on the device and every
    // kernel of an iteration does nothing once the solve has converged, so
    // iterations are launched in batches: as many as the previous solve took
    // (plus two), then the host reads the convergence flag once; only a solve
    // that needs more continues in smaller batches, each followed by a read.
    pq_status solve(const void* y, void* x, double tol) {
        void* r = vec(0);
        void* p = vec(1);
        void* Sp = vec(2);
        void* z = vec(5);
        double* cg = s.red_tmp + 8192;
        const int maxit = 2000;
        const double tol2 = tol * tol;
        pq_status rc;
        PQ_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(V), st));
        auto dot_into = [&](const void* a, const void* b, int mode) -> pq_status {
            k_cdot<R><<<G, kPvbThreads, 0, st>>>((const V*)a, (const V*)b, n, part,
                                                 mode == 0 || mode == 3 ? nullptr : cg + kCgDone);
            PQ_CHECK_LAUNCH();
            k_cg_scalar<<<1, 32, 0, st>>>(part, G, cg, mode, tol2);
            PQ_CHECK_LAUNCH();
            return PQ_OK;
        };
        auto axpy = [&](void* out, const void* x1, const void* x2, int slot, double sign) -> pq_status {
            k_cg_axpy<R><<<G, kPvbThreads, 0, st>>>((V*)out, (const V*)x1, (const V*)x2, n, cg, slot,
                                                    sign);
            PQ_CHECK_LAUNCH();
            return PQ_OK;
        };
        // start: r = y, z = M r, p = z
        if ((rc = lin(r, 1.0, y)) || (rc = dot_into(y, y, 0)) || (rc = Minv(r, z)) ||
            (rc = lin(p, 1.0, z)) || (rc = dot_into(r, z, 3)))
            return rc;
        gate = cg + kCgDone;
        int nodes = 0;
        auto iterate = [&]() -> pq_status {
            pq_status e;
            if ((e = S(p, Sp)) || (e = dot_into(p, Sp, 1)) || (e = axpy(x, x, p, kCgAlpha, 1.0)) ||
                (e = axpy(r, r, Sp, kCgAlpha, -1.0)) || (e = dot_into(r, r, 2)) || (e = Minv(r, z)) ||
                (e = dot_into(r, z, 4)) || (e = axpy(p, z, p, kCgBeta, 1.0)))
                return e;
            return PQ_OK;
        };
        // One iteration as a CUDA graph (captured on the state's private stream,
        // replayed on st): its 18 kernels cost one launch.  The self-checking
        // build synchronises after every launch and launches directly.
        cudaGraphExec_t ge = nullptr;
#ifndef PQ_BOUNDS_CHECK
        {
            if (!s.cap_stream)
                PQ_CUDA_TRY(cudaStreamCreateWithFlags(&s.cap_stream, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            const cudaStream_t st0 = st;
            const int64_t l0 = g_launches.load();
            PQ_CUDA_TRY(cudaStreamBeginCapture(s.cap_stream, cudaStreamCaptureModeRelaxed));
            st = s.cap_stream;
            const pq_status crc = iterate();
            st = st0;
            const cudaError_t ce = cudaStreamEndCapture(s.cap_stream, &g);
            nodes = (int)(g_launches.load() - l0);
            g_launches.fetch_sub(nodes);   // counted when they run
            if (crc) {
                if (g) cudaGraphDestroy(g);
                gate = nullptr;
                return crc;
            }
            PQ_CUDA_TRY(ce);
            const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            PQ_CUDA_TRY(ie);
        }
#endif
        struct GraphExec {
            cudaGraphExec_t& e;
            ~GraphExec() {
                if (e) cudaGraphExecDestroy(e);
            }
        } ge_owner{ge};
        auto step = [&]() -> pq_status {
            if (!ge) return iterate();
            PQ_CUDA_TRY(cudaGraphLaunch(ge, st));
            g_launches.fetch_add(nodes);
            return PQ_OK;
        };
        int launched = 0, batch = std::max(2, s.pvb_cg_pred);
        double flags[3];
        while (true) {
            for (int b = 0; b < batch && launched < maxit; ++b, ++launched)
                if ((rc = step())) {
                    gate = nullptr;
                    return rc;
                }
            PQ_CUDA_TRY(cudaMemcpyAsync(flags, cg + kCgDone, sizeof(flags), cudaMemcpyDeviceToHost, st));
            PQ_CUDA_TRY(cudaStreamSynchronize(st));
            if (flags[1] != 0.0) {
                gate = nullptr;
                set_error("pvB: conjugate gradients broke down");
                return PQ_ENUMERIC;
            }
            if (flags[0] != 0.0) {
                gate = nullptr;
                s.pvb_cg_pred = (int)flags[2] + 2;
                return PQ_OK;
            }
            if (launched >= maxit) break;
            batch = std::max(4, batch / 4);
        }
        gate = nullptr;
        set_error("pvB: conjugate gradients did not converge in %d iterations", maxit);
        return PQ_ENUMERIC;
    }
    // One Lanczos step of order K in the S inner product on the state's psi.
    pq_status sil(int K, double dt, double tol) {
        pq_status rc;
        void* a = s.psi;
        std::vector<void*> Vv(K);
        for (int k = 0; k < K; ++k) Vv[k] = (char*)s.V + (size_t)k * s.cap * sizeof(V);
        void* Hv = vec(3);
        void* Sw = vec(4);
        cd t;
        if ((rc = S(a, Sw)) || (rc = dot(a, Sw, &t))) return rc;
        const double beta0 = sqrt(std::max(t.real(), 0.0));
        if (!(beta0 > 0.0)) return PQ_OK;
        if ((rc = lin(Vv[0], 1.0 / beta0, a))) return rc;
        std::vector<double> alpha, beta;
        int keff = K;
        for (int k = 0; k < K; ++k) {
            cd al;
            if ((rc = H(Vv[k], Hv)) || (rc = dot(Vv[k], Hv, &al))) return rc;
            alpha.push_back(al.real());
            if (k == K - 1) break;
            cd hh;
            if ((rc = dot(Hv, Hv, &hh))) return rc;
            void* w = Vv[k + 1];
            if ((rc = solve(Hv, w, tol))) return rc;
            for (int pass = 0; pass < 2; ++pass) {
                if ((rc = S(w, Sw))) return rc;
                std::vector<cd> c(k + 1);
                for (int i = 0; i <= k; ++i)
                    if ((rc = dot(Vv[i], Sw, &c[i]))) return rc;
                for (int i = 0; i <= k; ++i)
                    if ((rc = lin(w, 1.0, w, -c[i], Vv[i]))) return rc;
            }
            cd ww;
            if ((rc = S(w, Sw)) || (rc = dot(w, Sw, &ww))) return rc;
            const double b = sqrt(std::max(ww.real(), 0.0));
            if (!(b > 1e-12 * sqrt(hh.real()) / std::max(1.0, s.pvb_smax))) {
                keff = k + 1;
                break;
            }
            beta.push_back(b);
            if ((rc = lin(w, 1.0 / b, w))) return rc;
        }
        keff = (int)alpha.size();
        // exp(-i T dt) e_1 by the host's symmetric eigensolver
        std::vector<double> Tm((size_t)keff * keff, 0.0), ev, Zm;
        for (int i = 0; i < keff; ++i) {
            Tm[(size_t)i * keff + i] = alpha[i];
            if (i + 1 < keff) Tm[(size_t)i * keff + i + 1] = Tm[(size_t)(i + 1) * keff + i] = beta[i];
        }
        if (jacobi_eigh(keff, Tm, ev, Zm) < 0) {
            set_error("pvB: tridiagonal eigensolver did not converge");
            return PQ_ENUMERIC;
        }
        std::vector<cd> cf(keff, 0.0);
        for (int j = 0; j < keff; ++j)
            for (int l = 0; l < keff; ++l)
                cf[j] += Zm[(size_t)j * keff + l] * std::exp(cd(0.0, -ev[l] * dt)) * Zm[l];
        if ((rc = lin(a, beta0 * cf[0], Vv[0]))) return rc;
        for (int j = 1; j < keff; ++j)
            if ((rc = lin(a, 1.0, a, beta0 * cf[j], Vv[j]))) return rc;
        return PQ_OK;
    }
};

template <typename R>
pq_status pvb_observe(State& s, double theta, cudaStream_t st) {
    Pvb<R> P(s, st);
    pq_status rc;
    if ((rc = P.count())) return rc;
    // C = <c|a> with c the B^dagger-mapped packet, as the observe kernel
    // computes it from the state's bra factors; norm = a^dagger S a; E = a^dagger H a / norm
    ObsRecord o{};
    o.t = s.t;
    o.n_active = P.n;
    void* Sa = P.vec(4);
    void* Ha = P.vec(3);
    cd nn, ee, cc;
    if ((rc = P.S(s.psi, Sa)) || (rc = P.dot(s.psi, Sa, &nn)) || (rc = P.H(s.psi, Ha)) ||
        (rc = P.dot(s.psi, Ha, &ee)))
        return rc;
    // bra on the active set: the packet with the bra factors, then <c|a>
    void* cvec = P.vec(0);
    const int Gp = grid_size() * 8;
    k_packet_bra<R><<<Gp, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap, s.lat,
                                        (const double2*)s.fac_bra64, (typename Cx<R>::T*)cvec);
    PQ_CHECK_LAUNCH();
    if ((rc = P.dot(cvec, s.psi, &cc))) return rc;
    o.c_re = cc.real();
    o.c_im = cc.imag();
    o.norm2 = nn.real();
    o.energy = nn.real() > 0 ? ee.real() / nn.real() : 0.0;
    // wasted: |a| < theta, counted on the host
    std::vector<typename Cx<R>::T> h((size_t)P.n);
    if (P.n > 0)
        PQ_CUDA_TRY(cudaMemcpyAsync(h.data(), s.psi, h.size() * sizeof(h[0]), cudaMemcpyDeviceToHost, st));
    PQ_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t wasted = 0;
    for (const auto& v : h) {
        const double re = v.x, im = v.y;
        if (!(re * re + im * im >= theta * theta)) ++wasted;
    }
    o.n_wasted = wasted;
    s.obs.push_back(o);
    s.obs_energy_pending = false;
    return PQ_OK;
}

}  // namespace

pq_status pvb_apply(State& s, const void* in, void* out, int prec, cudaStream_t st) {
    if (prec != s.prec) {
        set_error("pvB states apply H in their own precision");
        return PQ_EINVAL;
    }
    if (prec == PQ_FP64) {
        Pvb<double> P(s, st);
        return P.H(in, out);
    }
    Pvb<float> P(s, st);
    return P.H(in, out);
}

pq_status pvb_observe_current(State& s, double theta, cudaStream_t st) {
    return s.prec == PQ_FP64 ? pvb_observe<double>(s, theta, st) : pvb_observe<float>(s, theta, st);
}

pq_status pvb_propagate(State& s, const pq_prop_desc& d, int nsteps, cudaStream_t st) {
    if (d.integrator != PQ_SIL || d.sil_tol != 0.0) {
        set_error("pvB propagation provides fixed-order SIL only");
        return PQ_ENOTSUP;
    }
    pq_status rc = ensure_krylov(s, d.K);
    if (rc) return rc;
    const double tol = s.prec == PQ_FP64 ? 1e-13 : 1e-6;
    for (int n = 0; n < nsteps; ++n) {
        if (s.prec == PQ_FP64) {
            Pvb<double> P(s, st);
            if ((rc = P.count()) || (rc = P.sil(d.K, d.dt, tol))) return rc;
        } else {
            Pvb<float> P(s, st);
            if ((rc = P.count()) || (rc = P.sil(d.K, d.dt, tol))) return rc;
        }
        if ((rc = prune_launch(s, d.theta, d.radius, d.rel_excl, st))) return rc;
        s.t += d.dt;
        if ((rc = pvb_observe_current(s, d.theta, st))) return rc;
    }
    return PQ_OK;
}

}  // namespace pq
