// Pruned H.psi for DVR bases (Sec. 2.2.2 pruned sequential transform;
// Appendix: the transform is done one mode at a time over the fibres of the
// active set, J(i) in the paper's notation).  For a DVR Hamiltonian
// H = sum_k T^(k) + V with diagonal V (Sec. 2.1), the result equals
// P_A H P_A psi exactly:
//   out_I = sum_k sum_{j : I[k->j] in A} T^k_{i_k j} in_{I[k->j]} + V(x_I) in_I.
//
// GB300 layout: the active set is a rank/select bitmap over the lattice, so
// the members of any fibre are found with O(1) rank queries instead of the
// per-mode permutations of the paper.  Two kinds of work unit:
//  * inner pass: one warp per active "plane" (all digits but the last two
//    fixed).  A plane is one contiguous range of A; it is staged in shared
//    memory as a dense n[D-2] x n[D-1] tile (zero where inactive) and the
//    last two modes plus the on-the-fly SoP potential are applied; the output
//    is written once.
//  * outer pass, one per remaining mode k: one warp per fibre leader; the
//    n[k] rows of the fibre are staged as a dense tile and T^k is applied
//    along it; the output is accumulated (each point is in exactly one fibre
//    per mode, so there are no races).
// Zero-filled tiles give exactly the pruned product: inactive inputs
// contribute nothing and only active outputs are written.
//
// Kernel families, chosen per pass by launch_all:
//  * item-blocked (k_inner_q, k_outer_q): FP32, n[k] and n[D-1] <= 32;
//  * element-parallel (k_inner_ep, k_outer_ep): FP64, the same sizes;
//  * register-blocked, compact and generic tiles: other lengths up to 64;
//  * point-parallel (k_apply_point, k_pass_point): any mode longer than 64;
//  * generic single-mode passes (k_pass_row, k_pass_fibre): projected Weylets.
// A tabulated (non-SoP) diagonal potential is added per active point after
// the passes (k_add_grid_potential).
#include <type_traits>

#include "device_util.cuh"

namespace pq {

constexpr int kApplyThreads = 256;
constexpr size_t kSmemBudget = 200 * 1024;   // dynamic shared memory per block

template <typename R>
struct ApplyArgs {
    Lattice L;
    const uint64_t* bits;
    const uint32_t* off;
    const uint32_t* units;      // planes (inner) or fibre leaders (outer)
    const int64_t* nunits;
    const typename Cx<R>::T* in;
    typename Cx<R>::T* out;
    const double* in_scale;
    const int* skip;
    int skip_k;
    const R* T;                 // [D][kMaxN][kMaxN]
    const R* pot;               // [nterms][D][kMaxN] factor values (1 for identity)
    const R* potc;              // [nterms] term coefficients
    int nterms;
    int mode;                   // outer mode k (outer pass only)
    int wpb;                    // warps per block
    int64_t* cnt;               // state counters (bounds-check build)
    uint64_t units_cap;         // entries of the units array (bounds-check build)
    int ngroup[4];              // potential terms by tile modes touched (neither, D-2, D-1, both)
    const uint2* rowinfo;       // per-row (start, pattern) table, or null
    int full_gate;              // 1: run only on a dense set (>= half the lattice); -1: only below; 0: always
    const uint32_t* keys;       // sorted active linear indices (point-parallel pass)
    // generic single-mode pass (phase-space bases)
    const R* mat;               // n x n matrix of the pass (row stride kMaxN)
    double coef;                // result scale
    int accumulate;             // 1: out += coef * (M along mode) in;  0: out = ...
};

__device__ __forceinline__ uint64_t low_mask(int s) {
    return s >= 64 ? ~0ull : ((1ull << s) - 1ull);
}

// Dense-set gate: the item-blocked kernels and the dense-tile kernels of an
// FP32 H.psi are both launched, and the active-set size on the device selects
// which of them works (at least half the lattice active: the dense-tile
// kernels; the set can cross that size inside a device-driven propagation
// without the host seeing it).
template <typename A>
__device__ __forceinline__ bool gated_off(const A& a) {
    if (a.full_gate == 0) return false;
    const bool dense = 2 * a.cnt[CNT_NA] >= (int64_t)a.L.nfull;
    return dense != (a.full_gate > 0);
}

template <typename R>
__global__ void __launch_bounds__(kApplyThreads) k_apply_inner(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    // an active set that outgrew the capacity leaves positions beyond the
    // buffers: do nothing until the host sees the error
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int D = L.D, n2 = L.n[D - 2], nl = L.nlast, nt = a.nterms;
    // shared layout: per-warp tiles first (16-byte aligned), then tables
    const size_t tile_elems = (size_t)n2 * nl;
    V* tiles = reinterpret_cast<V*>(smem);
    uint64_t* rbits_all = reinterpret_cast<uint64_t*>(tiles + tile_elems * a.wpb);
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + (size_t)kMaxNTile * a.wpb);
    R* pref_all = reinterpret_cast<R*>(rstart_all + (size_t)kMaxNTile * a.wpb);
    R* Tq = pref_all + (size_t)kMaxTerms * a.wpb;   // [n2][n2]
    R* Tlt = Tq + n2 * n2;                          // [nl][nl], Tlt[ss][s] = T[s][ss]
    R* potq = Tlt + nl * nl;                        // [nt][n2]
    R* potl = potq + nt * n2;                       // [nt][nl]
    for (int i = threadIdx.x; i < n2 * n2; i += blockDim.x)
        Tq[i] = a.T[(size_t)(D - 2) * kMaxN * kMaxN + (i / n2) * kMaxN + (i % n2)];
    for (int i = threadIdx.x; i < nl * nl; i += blockDim.x) {
        const int ss = i / nl, s = i % nl;
        Tlt[i] = a.T[(size_t)(D - 1) * kMaxN * kMaxN + s * kMaxN + ss];
    }
    for (int i = threadIdx.x; i < nt * n2; i += blockDim.x)
        potq[i] = a.pot[((size_t)(i / n2) * D + (D - 2)) * kMaxN + (i % n2)];
    for (int i = threadIdx.x; i < nt * nl; i += blockDim.x)
        potl[i] = a.pot[((size_t)(i / nl) * D + (D - 1)) * kMaxN + (i % nl)];
    __syncthreads();

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    V* tile = tiles + tile_elems * w;
    uint64_t* rbits = rbits_all + (size_t)kMaxNTile * w;
    uint32_t* rstart = rstart_all + (size_t)kMaxNTile * w;
    R* pref = pref_all + (size_t)kMaxTerms * w;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
#ifdef PQ_BOUNDS_CHECK
    const uint64_t na = (uint64_t)a.cnt[CNT_NA];
#else
    const uint64_t na = 0;
#endif

    for (int64_t u = (int64_t)blockIdx.x * a.wpb + w; u < nunits;
         u += (int64_t)gridDim.x * a.wpb) {
        const uint32_t P = a.units[u];
        if (!pq_in_bounds(P, L.nplanes, 1, a.cnt)) continue;
        for (int j = lane; j < n2; j += 32) {
            const uint32_t r = P * (uint32_t)n2 + (uint32_t)j;
            const uint64_t b = row_bits(a.bits, r, nl);
            rbits[j] = b;
            rstart[j] = b ? rank_of(a.bits, a.off, (uint64_t)r * nl) : 0u;
        }
        for (int t = lane; t < nt; t += 32) {
            R p = a.potc[t];
            for (int k = 0; k < D - 2; ++k) {
                const int d = (int)((P / L.pstride[k]) % (uint32_t)L.n[k]);
                p *= a.pot[((size_t)t * D + k) * kMaxN + d];
            }
            pref[t] = p;
        }
        for (size_t e = lane; e < tile_elems; e += 32) tile[e] = cmake<R>(0, 0);
        __syncwarp();
        int jlo = n2, jhi = -1;
        for (int j = 0; j < n2; ++j) {
            const uint64_t b = rbits[j];
            if (!b) continue;
            jlo = min(jlo, j);
            jhi = j;
            const uint32_t st = rstart[j];
            for (int s = lane; s < nl; s += 32)
                if ((b >> s) & 1ull) {
                    const uint32_t pos = st + __popcll(b & low_mask(s));
                    if (!pq_in_bounds(pos, na, 2, a.cnt)) continue;
                    V v = a.in[pos];
                    v.x *= scale;
                    v.y *= scale;
                    tile[j * nl + s] = v;
                }
        }
        __syncwarp();
        for (int j = jlo; j <= jhi; ++j) {
            const uint64_t b = rbits[j];
            if (!b) continue;
            const uint32_t st = rstart[j];
            const int slo = __ffsll((long long)b) - 1, shi = 63 - __clzll((long long)b);
            const V* trow = tile + j * nl;
            for (int s = lane; s < nl; s += 32) {
                if (!((b >> s) & 1ull)) continue;
                R ax = 0, ay = 0;
                const R* tq = Tq + j * n2;
                for (int jj = jlo; jj <= jhi; ++jj) {
                    const R t = tq[jj];
                    const V c = tile[jj * nl + s];
                    ax += t * c.x;
                    ay += t * c.y;
                }
                for (int ss = slo; ss <= shi; ++ss) {
                    const R t = Tlt[ss * nl + s];
                    const V c = trow[ss];
                    ax += t * c.x;
                    ay += t * c.y;
                }
                R vv = 0;
                for (int t = 0; t < nt; ++t) vv += pref[t] * potq[t * n2 + j] * potl[t * nl + s];
                const V c = trow[s];
                ax += vv * c.x;
                ay += vv * c.y;
                const uint32_t pos = st + __popcll(b & low_mask(s));
                if (pq_in_bounds(pos, na, 3, a.cnt)) a.out[pos] = cmake<R>(ax, ay);
            }
        }
        __syncwarp();
    }
}

template <typename R>
__global__ void __launch_bounds__(kApplyThreads) k_apply_outer(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    // an active set that outgrew the capacity leaves positions beyond the
    // buffers: do nothing until the host sees the error
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int k = a.mode, nk = L.n[k], nl = L.nlast;
    const uint32_t rs = L.rstride[k];
    const size_t tile_elems = (size_t)nk * nl;
    V* tiles = reinterpret_cast<V*>(smem);
    uint64_t* rbits_all = reinterpret_cast<uint64_t*>(tiles + tile_elems * a.wpb);
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + (size_t)kMaxNTile * a.wpb);
    R* Tk = reinterpret_cast<R*>(rstart_all + (size_t)kMaxNTile * a.wpb);   // [nk][nk]
    for (int i = threadIdx.x; i < nk * nk; i += blockDim.x)
        Tk[i] = a.T[(size_t)k * kMaxN * kMaxN + (i / nk) * kMaxN + (i % nk)];
    __syncthreads();

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    V* tile = tiles + tile_elems * w;
    uint64_t* rbits = rbits_all + (size_t)kMaxNTile * w;
    uint32_t* rstart = rstart_all + (size_t)kMaxNTile * w;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
#ifdef PQ_BOUNDS_CHECK
    const uint64_t na = (uint64_t)a.cnt[CNT_NA];
#else
    const uint64_t na = 0;
#endif

    for (int64_t u = (int64_t)blockIdx.x * a.wpb + w; u < nunits;
         u += (int64_t)gridDim.x * a.wpb) {
        if (!pq_in_bounds((uint64_t)u, a.units_cap, 11, a.cnt)) continue;
        const uint32_t r0 = a.units[u];
        if (!pq_in_bounds(r0, L.nrows, 4, a.cnt)) continue;
        const int i0 = (int)((r0 / rs) % (uint32_t)nk);
        for (int j = lane; j < nk; j += 32) {
            uint64_t b = 0;
            uint32_t st = 0;
            if (j >= i0) {
                const uint32_t r = r0 + (uint32_t)(j - i0) * rs;
                if (!pq_in_bounds(r, L.nrows, 12, a.cnt)) continue;
                if (!pq_in_bounds(((uint64_t)r * nl + nl - 1) >> 6, L.nwords, 13, a.cnt)) continue;
                b = row_bits(a.bits, r, nl);
                if (b) st = rank_of(a.bits, a.off, (uint64_t)r * nl);
            }
            rbits[j] = b;
            rstart[j] = st;
        }
        for (size_t e = lane; e < tile_elems; e += 32) tile[e] = cmake<R>(0, 0);
        __syncwarp();
        int jhi = -1;
        for (int j = i0; j < nk; ++j) {
            const uint64_t b = rbits[j];
            if (!b) continue;
            jhi = j;
            const uint32_t st = rstart[j];
            for (int s = lane; s < nl; s += 32)
                if ((b >> s) & 1ull) {
                    const uint32_t pos = st + __popcll(b & low_mask(s));
                    if (!pq_in_bounds(pos, na, 5, a.cnt)) continue;
                    if (!pq_in_bounds((uint64_t)(j * nl + s), tile_elems, 14, a.cnt)) continue;
                    V v = a.in[pos];
                    v.x *= scale;
                    v.y *= scale;
                    tile[j * nl + s] = v;
                }
        }
        __syncwarp();
        for (int j = i0; j <= jhi; ++j) {
            const uint64_t b = rbits[j];
            if (!b) continue;
            const uint32_t st = rstart[j];
            const R* tk = Tk + j * nk;
            for (int s = lane; s < nl; s += 32) {
                if (!((b >> s) & 1ull)) continue;
                R ax = 0, ay = 0;
                if (!pq_in_bounds((uint64_t)(jhi * nl + s), tile_elems, 15, a.cnt)) continue;
                if (!pq_in_bounds((uint64_t)(j * nk + jhi), (uint64_t)nk * nk, 16, a.cnt)) continue;
                for (int jj = i0; jj <= jhi; ++jj) {
                    const R t = tk[jj];
                    const V c = tile[jj * nl + s];
                    ax += t * c.x;
                    ay += t * c.y;
                }
                const uint32_t pos = st + __popcll(b & low_mask(s));
                if (!pq_in_bounds(pos, na, 6, a.cnt)) continue;
                V* o = a.out + pos;
                V ov = *o;
                ov.x += ax;
                ov.y += ay;
                *o = ov;
            }
        }
        __syncwarp();
    }
}


// ------------------------------------------------------------------------
// Register-blocked fibre kernels for compile-time fibre lengths (the common
// 16/24/32-point modes).  A warp still owns one plane / one fibre, but lane s
// keeps the whole column s of the fibre tile in registers, and each output
// row j is a dot product of that column with row j of the 1D operator, read
// as vectorised shared-memory broadcasts (4 entries per load).  This removes
// the per-FMA shared-memory traffic of the generic kernels above.
// Requires n[D-1] <= 32 (one lane per last-mode point).

// four consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void ld4(const float* p, float& a, float& b, float& c, float& d) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double& a, double& b, double& c, double& d) {
    const double2 u = *reinterpret_cast<const double2*>(p);
    const double2 v = *reinterpret_cast<const double2*>(p + 2);
    a = u.x; b = u.y; c = v.x; d = v.y;
}

// acc += sum_jj t[jj] * (cx[jj], cy[jj]) over jj in [0, N), with whole
// 8-entry chunks outside [jlo, jhi] skipped (warp-uniform branch).
template <typename R, int N>
__device__ __forceinline__ void row_dot(const R* __restrict__ t, const R (&cx)[N],
                                        const R (&cy)[N], int jlo, int jhi, R& ax, R& ay) {
#pragma unroll
    for (int c = 0; c < N; c += 8) {
        if (c + 8 <= jlo || c > jhi) continue;
#pragma unroll
        for (int q = 0; q < 8 && c + q < N; q += 4) {
            R t0, t1, t2, t3;
            ld4(t + c + q, t0, t1, t2, t3);
            ax += t0 * cx[c + q] + t1 * cx[c + q + 1] + t2 * cx[c + q + 2] + t3 * cx[c + q + 3];
            ay += t0 * cy[c + q] + t1 * cy[c + q + 1] + t2 * cy[c + q + 2] + t3 * cy[c + q + 3];
        }
    }
}

template <typename R, int NK>
__global__ void __launch_bounds__(kApplyThreads) k_apply_outer_reg(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int k = a.mode, nl = L.nlast;
    const uint32_t rs = L.rstride[k];
    R* Tk = reinterpret_cast<R*>(smem);                              // [NK][NK]
    uint64_t* rbits_all = reinterpret_cast<uint64_t*>(Tk + NK * NK);
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + NK * a.wpb);
    for (int i = threadIdx.x; i < NK * NK; i += blockDim.x)
        Tk[i] = a.T[(size_t)k * kMaxN * kMaxN + (i / NK) * kMaxN + (i % NK)];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    uint64_t* rbits = rbits_all + NK * w;
    uint32_t* rstart = rstart_all + NK * w;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
    const uint64_t lmask = (1ull << lane) - 1ull;
    const bool lane_ok = lane < nl;
    for (int64_t u = (int64_t)blockIdx.x * a.wpb + w; u < nunits;
         u += (int64_t)gridDim.x * a.wpb) {
        const uint32_t r0 = a.units[u];
        const int i0 = (int)((r0 / rs) % (uint32_t)NK);
        for (int j = lane; j < NK; j += 32) {
            uint64_t b = 0;
            uint32_t st = 0;
            if (j >= i0) {
                const uint32_t r = r0 + (uint32_t)(j - i0) * rs;
                if (a.rowinfo) {
                    const uint2 ri = a.rowinfo[r];
                    st = ri.x;
                    b = ri.y;
                } else {
                    b = row_bits(a.bits, r, nl);
                    if (b) st = rank_of(a.bits, a.off, (uint64_t)r * nl);
                }
            }
            rbits[j] = b;
            rstart[j] = st;
        }
        __syncwarp();
        R cx[NK], cy[NK];
        int jhi = i0;
#pragma unroll
        for (int jj = 0; jj < NK; ++jj) {
            const uint64_t b = rbits[jj];
            if (b) jhi = jj;
            R x = 0, y = 0;
            if (lane_ok && ((b >> lane) & 1ull)) {
                const V v = a.in[rstart[jj] + __popcll(b & lmask)];
                x = v.x * scale;
                y = v.y * scale;
            }
            cx[jj] = x;
            cy[jj] = y;
        }
        for (int j = i0; j <= jhi; ++j) {
            const uint64_t b = rbits[j];
            if (!b) continue;
            R ax = 0, ay = 0;
            row_dot<R, NK>(Tk + j * NK, cx, cy, i0, jhi, ax, ay);
            if (lane_ok && ((b >> lane) & 1ull)) {
                V* o = a.out + rstart[j] + __popcll(b & lmask);
                V ov = *o;
                ov.x += ax;
                ov.y += ay;
                *o = ov;
            }
        }
        __syncwarp();
    }
}

// Inner pass, register-blocked: modes D-2 (column dot products, as above) and
// D-1 (row dot products: lane s keeps row s of T^(D-1) in registers and reads
// the tile row as broadcasts), plus the potential split by the tile modes each
// term touches: V(j,s) = f(j) + g(s) + sum_{both} A_t(j) B_t(s), where f holds
// the terms constant in s (including plane constants), g those constant in j.
template <typename R, int N2, int NL>
__global__ void __launch_bounds__(kApplyThreads) k_apply_inner_reg(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int D = L.D, nt = a.nterms;
    const int g1 = a.ngroup[0], g2 = g1 + a.ngroup[1], g3 = g2 + a.ngroup[2];   // group starts
    // shared: Tq [N2][N2], then per warp: tile [N2][NL] (V), rbits [N2], rstart [N2],
    // pref [kMaxTerms], f [N2]
    R* Tq = reinterpret_cast<R*>(smem);
    V* tiles = reinterpret_cast<V*>(Tq + N2 * N2);
    uint64_t* rbits_all = reinterpret_cast<uint64_t*>(tiles + N2 * NL * a.wpb);
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + N2 * a.wpb);
    R* pref_all = reinterpret_cast<R*>(rstart_all + N2 * a.wpb);
    R* f_all = pref_all + kMaxTerms * a.wpb;
    for (int i = threadIdx.x; i < N2 * N2; i += blockDim.x)
        Tq[i] = a.T[(size_t)(D - 2) * kMaxN * kMaxN + (i / N2) * kMaxN + (i % N2)];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    const int ls = lane < NL ? lane : NL - 1;
    // row ls of T^(D-1) and the mode-(D-1) potential factors in registers
    R tl[NL];
#pragma unroll
    for (int ss = 0; ss < NL; ++ss) tl[ss] = a.T[(size_t)(D - 1) * kMaxN * kMaxN + ls * kMaxN + ss];
    V* tile = tiles + N2 * NL * w;
    uint64_t* rbits = rbits_all + N2 * w;
    uint32_t* rstart = rstart_all + N2 * w;
    R* pref = pref_all + kMaxTerms * w;
    R* fj = f_all + N2 * w;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
    const uint64_t lmask = (1ull << lane) - 1ull;
    const bool lane_ok = lane < NL;
    for (int64_t u = (int64_t)blockIdx.x * a.wpb + w; u < nunits;
         u += (int64_t)gridDim.x * a.wpb) {
        const uint32_t P = a.units[u];
        for (int j = lane; j < N2; j += 32) {
            const uint32_t r = P * (uint32_t)N2 + (uint32_t)j;
            if (a.rowinfo) {
                const uint2 ri = a.rowinfo[r];
                rbits[j] = ri.y;
                rstart[j] = ri.x;
            } else {
                const uint64_t b = row_bits(a.bits, r, NL);
                rbits[j] = b;
                rstart[j] = b ? rank_of(a.bits, a.off, (uint64_t)r * NL) : 0u;
            }
        }
        for (int t = lane; t < nt; t += 32) {
            R p = a.potc[t];
            for (int k = 0; k < D - 2; ++k) {
                const int d = (int)((P / L.pstride[k]) % (uint32_t)L.n[k]);
                p *= a.pot[((size_t)t * D + k) * kMaxN + d];
            }
            pref[t] = p;
        }
        __syncwarp();
        // f(j): terms constant along the last mode
        for (int j = lane; j < N2; j += 32) {
            R f = 0;
            for (int t = 0; t < g1; ++t) f += pref[t];
            for (int t = g1; t < g2; ++t) f += pref[t] * a.pot[((size_t)t * D + D - 2) * kMaxN + j];
            fj[j] = f;
        }
        // g(s): terms constant along mode D-2
        R gs = 0;
        for (int t = g2; t < g3; ++t) gs += pref[t] * a.pot[((size_t)t * D + D - 1) * kMaxN + ls];
        // column s of the plane in registers, and the plane in shared memory
        R cx[N2], cy[N2];
        int jlo = N2, jhi = -1;
#pragma unroll
        for (int jj = 0; jj < N2; ++jj) {
            const uint64_t b = rbits[jj];
            if (b) {
                jlo = min(jlo, jj);
                jhi = jj;
            }
            R x = 0, y = 0;
            if (lane_ok && ((b >> lane) & 1ull)) {
                const V v = a.in[rstart[jj] + __popcll(b & lmask)];
                x = v.x * scale;
                y = v.y * scale;
            }
            cx[jj] = x;
            cy[jj] = y;
            if (lane_ok) tile[jj * NL + lane] = cmake<R>(x, y);
        }
        __syncwarp();
        for (int j = jlo; j <= jhi; ++j) {
            const uint64_t b = rbits[j];
            if (!b) continue;
            R ax = 0, ay = 0;
            row_dot<R, N2>(Tq + j * N2, cx, cy, jlo, jhi, ax, ay);   // mode D-2
            const V* trow = tile + j * NL;                            // mode D-1
            const int slo = (__ffsll((long long)b) - 1) & ~1;
            const int shi = 63 - __clzll((long long)b);
#pragma unroll
            for (int ss = 0; ss < NL; ss += 2) {
                if (ss + 1 < slo || ss > shi) continue;
                R x0, y0, x1, y1;
                ld4(reinterpret_cast<const R*>(trow + ss), x0, y0, x1, y1);
                ax += tl[ss] * x0 + tl[ss + 1] * x1;
                ay += tl[ss] * y0 + tl[ss + 1] * y1;
            }
            if (lane_ok && ((b >> lane) & 1ull)) {
                R vv = fj[j] + gs;
                for (int t = g3; t < nt; ++t)
                    vv += pref[t] * a.pot[((size_t)t * D + D - 2) * kMaxN + j] *
                          a.pot[((size_t)t * D + D - 1) * kMaxN + lane];
                const V c = trow[lane];
                ax += vv * c.x;
                ay += vv * c.y;
                a.out[rstart[j] + __popcll(b & lmask)] = cmake<R>(ax, ay);
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------
// Compact fibre kernels (used whenever n[D-1] <= 32).  The fibre tiles of a
// pruned set are sparse (for a 6D ellipsoid about 15-20 % of the n[k] x
// n[D-1] tile is active), so each warp first compacts the fibre's active rows
// (ballot), gathers only those rows into shared memory, and runs the dot
// products over active rows only: the work per output is the number of active
// partners, not the fibre length.  Lane s owns last-mode point s.

template <typename R>
__global__ void __launch_bounds__(kApplyThreads) k_apply_outer_cmp(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int k = a.mode, nk = L.n[k], nl = L.nlast;
    const uint32_t rs = L.rstride[k];
    // per warp: xin [nk][32] V, rbits [64], rstart [64], rowj [64], trow [64] R
    V* tiles = reinterpret_cast<V*>(smem);
    uint64_t* rbits_all = reinterpret_cast<uint64_t*>(tiles + (size_t)nk * 32 * a.wpb);
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + kMaxNTile * a.wpb);
    int* rowj_all = reinterpret_cast<int*>(rstart_all + kMaxNTile * a.wpb);
    R* trow_all = reinterpret_cast<R*>(rowj_all + kMaxNTile * a.wpb);
    R* Tk = trow_all + kMaxNTile * a.wpb;                       // [nk][nk]
    for (int i = threadIdx.x; i < nk * nk; i += blockDim.x)
        Tk[i] = a.T[(size_t)k * kMaxN * kMaxN + (i / nk) * kMaxN + (i % nk)];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    V* xin = tiles + (size_t)nk * 32 * w;
    uint64_t* rbits = rbits_all + kMaxNTile * w;
    uint32_t* rstart = rstart_all + kMaxNTile * w;
    int* rowj = rowj_all + kMaxNTile * w;
    R* trow = trow_all + kMaxNTile * w;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
    const uint64_t lmask = (1ull << lane) - 1ull;
    const int64_t ustep = (int64_t)gridDim.x * a.wpb;
    int64_t u = (int64_t)blockIdx.x * a.wpb + w;
    uint32_t r0n = u < nunits ? a.units[u] : 0u;
    for (; u < nunits; u += ustep) {
        const uint32_t r0 = r0n;
        if (u + ustep < nunits) r0n = a.units[u + ustep];   // next fibre, in flight
        const int i0 = (int)((r0 / rs) % (uint32_t)nk);
        // active rows of the fibre, compacted in order of j
        int na = 0;
        for (int jb = 0; jb < nk; jb += 32) {
            const int j = jb + lane;
            uint64_t b = 0;
            uint32_t st = 0;
            if (j < nk && j >= i0) {
                const uint32_t r = r0 + (uint32_t)(j - i0) * rs;
                if (a.rowinfo) {
                    const uint2 ri = a.rowinfo[r];
                    st = ri.x;
                    b = ri.y;
                } else {
                    b = row_bits(a.bits, r, nl);
                    if (b) st = rank_of(a.bits, a.off, (uint64_t)r * nl);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, b != 0);
            if (b) {
                const int slot = na + __popc(m & (unsigned)lmask);
                rbits[slot] = b;
                rstart[slot] = st;
                rowj[slot] = j;
            }
            na += __popc(m);
        }
        __syncwarp();
        // inputs and the outputs accumulated so far, all loads in flight at once
#pragma unroll 4
        for (int v = 0; v < na; ++v) {
            const uint64_t b = rbits[v];
            V x = cmake<R>(0, 0);
            if ((b >> lane) & 1ull) {
                x = a.in[rstart[v] + __popcll(b & lmask)];
                x.x *= scale;
                x.y *= scale;
            }
            xin[v * 32 + lane] = x;
        }
        __syncwarp();
        for (int uo = 0; uo < na; ++uo) {
            const int j = rowj[uo];
            const R* tj = Tk + j * nk;
            for (int v = lane; v < na; v += 32) trow[v] = tj[rowj[v]];
            __syncwarp();
            const uint64_t b = rbits[uo];
            if ((b >> lane) & 1ull) {
                V* o = a.out + rstart[uo] + __popcll(b & lmask);
                V ov = *o;                                // in flight during the dot product
                R ax = 0, ay = 0;
                for (int v = 0; v < na; ++v) {
                    const R t = trow[v];
                    const V c = xin[v * 32 + lane];
                    ax += t * c.x;
                    ay += t * c.y;
                }
                ov.x += ax;
                ov.y += ay;
                *o = ov;
            }
            __syncwarp();
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kApplyThreads) k_apply_inner_cmp(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int D = L.D, n2 = L.n[D - 2], nl = L.nlast, nt = a.nterms;
    const int g1 = a.ngroup[0], g2 = g1 + a.ngroup[1], g3 = g2 + a.ngroup[2];
    // per warp: tile [n2][32] V, rbits [64], rstart [64], rowj [64], trow [64] R,
    // pref [kMaxTerms] R, fj [64] R; shared: Tq [n2][n2], Tlt [nl][32]
    V* tiles = reinterpret_cast<V*>(smem);
    uint64_t* rbits_all = reinterpret_cast<uint64_t*>(tiles + (size_t)n2 * 32 * a.wpb);
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + kMaxNTile * a.wpb);
    int* rowj_all = reinterpret_cast<int*>(rstart_all + kMaxNTile * a.wpb);
    R* trow_all = reinterpret_cast<R*>(rowj_all + kMaxNTile * a.wpb);
    R* pref_all = trow_all + kMaxNTile * a.wpb;
    R* fj_all = pref_all + kMaxTerms * a.wpb;
    R* Tq = fj_all + kMaxNTile * a.wpb;                         // [n2][n2]
    R* Tlt = Tq + n2 * n2;                                  // [nl][32]: Tlt[ss][s] = T[s][ss]
    for (int i = threadIdx.x; i < n2 * n2; i += blockDim.x)
        Tq[i] = a.T[(size_t)(D - 2) * kMaxN * kMaxN + (i / n2) * kMaxN + (i % n2)];
    for (int i = threadIdx.x; i < nl * 32; i += blockDim.x) {
        const int ss = i / 32, sl = i % 32;
        Tlt[i] = sl < nl ? a.T[(size_t)(D - 1) * kMaxN * kMaxN + sl * kMaxN + ss] : (R)0;
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    V* tile = tiles + (size_t)n2 * 32 * w;
    uint64_t* rbits = rbits_all + kMaxNTile * w;
    uint32_t* rstart = rstart_all + kMaxNTile * w;
    int* rowj = rowj_all + kMaxNTile * w;
    R* trow = trow_all + kMaxNTile * w;
    R* pref = pref_all + kMaxTerms * w;
    R* fj = fj_all + kMaxNTile * w;
    const int ls = lane < nl ? lane : nl - 1;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
    const uint64_t lmask = (1ull << lane) - 1ull;
    for (int64_t u = (int64_t)blockIdx.x * a.wpb + w; u < nunits;
         u += (int64_t)gridDim.x * a.wpb) {
        const uint32_t P = a.units[u];
        int na = 0;
        for (int jb = 0; jb < n2; jb += 32) {
            const int j = jb + lane;
            uint64_t b = 0;
            uint32_t st = 0;
            if (j < n2) {
                const uint32_t r = P * (uint32_t)n2 + (uint32_t)j;
                if (a.rowinfo) {
                    const uint2 ri = a.rowinfo[r];
                    st = ri.x;
                    b = ri.y;
                } else {
                    b = row_bits(a.bits, r, nl);
                    if (b) st = rank_of(a.bits, a.off, (uint64_t)r * nl);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, b != 0);
            if (b) {
                const int slot = na + __popc(m & (unsigned)lmask);
                rbits[slot] = b;
                rstart[slot] = st;
                rowj[slot] = j;
            }
            na += __popc(m);
        }
        for (int t = lane; t < nt; t += 32) {
            R p = a.potc[t];
            for (int k = 0; k < D - 2; ++k) {
                const int d = (int)((P / L.pstride[k]) % (uint32_t)L.n[k]);
                p *= a.pot[((size_t)t * D + k) * kMaxN + d];
            }
            pref[t] = p;
        }
        __syncwarp();
        for (int v = lane; v < na; v += 32) {   // f(j): terms constant along the last mode
            const int j = rowj[v];
            R f = 0;
            for (int t = 0; t < g1; ++t) f += pref[t];
            for (int t = g1; t < g2; ++t) f += pref[t] * a.pot[((size_t)t * D + D - 2) * kMaxN + j];
            fj[v] = f;
        }
        R gs = 0;                                 // g(s): terms constant along mode D-2
        for (int t = g2; t < g3; ++t) gs += pref[t] * a.pot[((size_t)t * D + D - 1) * kMaxN + ls];
#pragma unroll 4
        for (int v = 0; v < na; ++v) {
            const uint64_t b = rbits[v];
            V x = cmake<R>(0, 0);
            if ((b >> lane) & 1ull) {
                x = a.in[rstart[v] + __popcll(b & lmask)];
                x.x *= scale;
                x.y *= scale;
            }
            tile[v * 32 + lane] = x;
        }
        __syncwarp();
        for (int uo = 0; uo < na; ++uo) {
            const int j = rowj[uo];
            const R* tj = Tq + j * n2;
            for (int v = lane; v < na; v += 32) trow[v] = tj[rowj[v]];
            __syncwarp();
            const uint64_t b = rbits[uo];
            if ((b >> lane) & 1ull) {
                R ax = 0, ay = 0;
                for (int v = 0; v < na; ++v) {            // mode D-2
                    const R t = trow[v];
                    const V c = tile[v * 32 + lane];
                    ax += t * c.x;
                    ay += t * c.y;
                }
                const V* rowv = tile + uo * 32;           // mode D-1
                const int slo = __ffsll((long long)b) - 1, shi = 63 - __clzll((long long)b);
                for (int ss = slo; ss <= shi; ++ss) {
                    const R t = Tlt[ss * 32 + lane];
                    const V c = rowv[ss];
                    ax += t * c.x;
                    ay += t * c.y;
                }
                R vv = fj[uo] + gs;
                for (int t = g3; t < nt; ++t)
                    vv += pref[t] * a.pot[((size_t)t * D + D - 2) * kMaxN + j] *
                          a.pot[((size_t)t * D + D - 1) * kMaxN + lane];
                const V c = rowv[lane];
                ax += vv * c.x;
                ay += vv * c.y;
                a.out[rstart[uo] + __popcll(b & lmask)] = cmake<R>(ax, ay);
            }
            __syncwarp();
        }
    }
}

template <typename R>
static size_t smem_outer_cmp(int nk, int wpb) {
    const size_t esz = sizeof(R);
    return (size_t)wpb * ((size_t)nk * 32 * 2 * esz + kMaxNTile * (8 + 4 + 4 + esz)) + (size_t)nk * nk * esz;
}
template <typename R>
static size_t smem_inner_cmp(int n2, int nl, int wpb) {
    const size_t esz = sizeof(R);
    return (size_t)wpb * ((size_t)n2 * 32 * 2 * esz + kMaxNTile * (8 + 4 + 4 + esz) + kMaxTerms * esz +
                          kMaxNTile * esz) +
           ((size_t)n2 * n2 + (size_t)nl * 32) * esz;
}

// ------------------------------------------------------------------------
// Generic single-mode passes for SoP Hamiltonians with dense 1D factors
// (projected Weylets, Sec. 2.4; pruned sequential transform, Sec. 2.2.2):
//   out (+)= coef * P_A (M along mode k) in.
// Last mode: one warp per active row (the row is contiguous in A).  Other
// modes: one warp per fibre leader, the fibre staged as a dense tile.

template <typename R>
__global__ void __launch_bounds__(kApplyThreads) k_pass_row(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int nl = L.nlast;
    R* Mt = reinterpret_cast<R*>(smem);                    // [nl][nl], Mt[ss][s] = M[s][ss]
    V* xrow_all = reinterpret_cast<V*>(Mt + ((nl * nl + 1) & ~1));
    for (int i = threadIdx.x; i < nl * nl; i += blockDim.x) {
        const int ss = i / nl, sl = i % nl;
        Mt[i] = a.mat[sl * kMaxN + ss];
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    V* xrow = xrow_all + kMaxNTile * w;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const R coef = (R)a.coef;
    const int64_t nunits = *a.nunits;
    for (int64_t u = (int64_t)blockIdx.x * a.wpb + w; u < nunits;
         u += (int64_t)gridDim.x * a.wpb) {
        const uint32_t r = a.units[u];
        const uint64_t b = row_bits(a.bits, r, nl);
        const uint32_t st = rank_of(a.bits, a.off, (uint64_t)r * nl);
        for (int s = lane; s < nl; s += 32) {
            V x = cmake<R>(0, 0);
            if ((b >> s) & 1ull) {
                x = a.in[st + __popcll(b & low_mask(s))];
                x.x *= scale;
                x.y *= scale;
            }
            xrow[s] = x;
        }
        __syncwarp();
        const int slo = __ffsll((long long)b) - 1, shi = 63 - __clzll((long long)b);
        for (int s = lane; s < nl; s += 32) {
            if (!((b >> s) & 1ull)) continue;
            R ax = 0, ay = 0;
            for (int ss = slo; ss <= shi; ++ss) {
                const R t = Mt[ss * nl + s];
                const V c = xrow[ss];
                ax += t * c.x;
                ay += t * c.y;
            }
            V* o = a.out + st + __popcll(b & low_mask(s));
            V y = cmake<R>(coef * ax, coef * ay);
            if (a.accumulate) {
                const V ov = *o;
                y.x += ov.x;
                y.y += ov.y;
            }
            *o = y;
        }
        __syncwarp();
    }
}

template <typename R>
__global__ void __launch_bounds__(kApplyThreads) k_pass_fibre(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int k = a.mode, nk = L.n[k], nl = L.nlast;
    const uint32_t rs = L.rstride[k];
    const size_t tile_elems = (size_t)nk * nl;
    V* tiles = reinterpret_cast<V*>(smem);
    uint64_t* rbits_all = reinterpret_cast<uint64_t*>(tiles + tile_elems * a.wpb);
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + (size_t)kMaxNTile * a.wpb);
    R* Mk = reinterpret_cast<R*>(rstart_all + (size_t)kMaxNTile * a.wpb);   // [nk][nk]
    for (int i = threadIdx.x; i < nk * nk; i += blockDim.x) Mk[i] = a.mat[(i / nk) * kMaxN + (i % nk)];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    V* tile = tiles + tile_elems * w;
    uint64_t* rbits = rbits_all + (size_t)kMaxNTile * w;
    uint32_t* rstart = rstart_all + (size_t)kMaxNTile * w;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const R coef = (R)a.coef;
    const int64_t nunits = *a.nunits;
    for (int64_t u = (int64_t)blockIdx.x * a.wpb + w; u < nunits;
         u += (int64_t)gridDim.x * a.wpb) {
        const uint32_t r0 = a.units[u];
        const int i0 = (int)((r0 / rs) % (uint32_t)nk);
        for (int j = lane; j < nk; j += 32) {
            uint64_t b = 0;
            uint32_t st = 0;
            if (j >= i0) {
                const uint32_t r = r0 + (uint32_t)(j - i0) * rs;
                b = row_bits(a.bits, r, nl);
                if (b) st = rank_of(a.bits, a.off, (uint64_t)r * nl);
            }
            rbits[j] = b;
            rstart[j] = st;
        }
        for (size_t e = lane; e < tile_elems; e += 32) tile[e] = cmake<R>(0, 0);
        __syncwarp();
        int jhi = -1;
        for (int j = i0; j < nk; ++j) {
            const uint64_t b = rbits[j];
            if (!b) continue;
            jhi = j;
            const uint32_t st = rstart[j];
            for (int s = lane; s < nl; s += 32)
                if ((b >> s) & 1ull) {
                    V v = a.in[st + __popcll(b & low_mask(s))];
                    v.x *= scale;
                    v.y *= scale;
                    tile[j * nl + s] = v;
                }
        }
        __syncwarp();
        for (int j = i0; j <= jhi; ++j) {
            const uint64_t b = rbits[j];
            if (!b) continue;
            const uint32_t st = rstart[j];
            const R* mj = Mk + j * nk;
            for (int s = lane; s < nl; s += 32) {
                if (!((b >> s) & 1ull)) continue;
                R ax = 0, ay = 0;
                for (int jj = i0; jj <= jhi; ++jj) {
                    const R t = mj[jj];
                    const V c = tile[jj * nl + s];
                    ax += t * c.x;
                    ay += t * c.y;
                }
                V* o = a.out + st + __popcll(b & low_mask(s));
                V y = cmake<R>(coef * ax, coef * ay);
                if (a.accumulate) {
                    const V ov = *o;
                    y.x += ov.x;
                    y.y += ov.y;
                }
                *o = y;
            }
        }
        __syncwarp();
    }
}

template <typename R>
__global__ void k_zero(typename Cx<R>::T* out, const int64_t* na, const int* skip, int skip_k) {
    if (skip && *skip <= skip_k) return;
    const int64_t n = *na;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        out[p] = cmake<R>(0, 0);
}

// Point-parallel single-mode pass (lattices with a mode longer than 64):
// out_I (+)= coef * sum_j M[i_k][j] in_{I[k->j]} over the active j, one thread
// per active point.
template <typename R>
__global__ void __launch_bounds__(256) k_pass_point(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    const Lattice& L = a.L;
    const int k = a.mode, nk = L.n[k];
    const uint32_t sk = L.stride[k];
    const int64_t n = a.cnt[CNT_NA];
    const R scale = (a.in_scale ? (R)(*a.in_scale) : (R)1) * (R)a.coef;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = a.keys[p];
        const int d = (int)((key / sk) % (uint32_t)nk);
        const uint32_t base = key - (uint32_t)d * sk;
        const R* mrow = a.mat + (size_t)d * kMaxN;
        R ax = 0, ay = 0;
        for (int j = 0; j < nk; ++j) {
            const uint32_t q = base + (uint32_t)j * sk;
            if (!bit_test(a.bits, q)) continue;
            const uint32_t pos = rank_of(a.bits, a.off, q);
            if (!pq_in_bounds(pos, (uint64_t)n, 30, a.cnt)) continue;
            const V x = a.in[pos];
            ax += mrow[j] * x.x;
            ay += mrow[j] * x.y;
        }
        V y = cmake<R>(scale * ax, scale * ay);
        if (a.accumulate) {
            const V o = a.out[p];
            y.x += o.x;
            y.y += o.y;
        }
        a.out[p] = y;
    }
}

template <typename R>
static pq_status launch_pass(const State& s, ApplyArgs<R> a, int mode, int mat, const void* in,
                             void* out, const double* in_scale, double coef, int accumulate,
                             cudaStream_t st) {
    const Lattice& L = s.lat;
    const size_t esz = sizeof(R);
    a.in = (const typename Cx<R>::T*)in;
    a.out = (typename Cx<R>::T*)out;
    a.in_scale = in_scale;
    a.mat = (sizeof(R) == 8 ? (const R*)s.gmat64 : (const R*)s.gmat32) + (size_t)mat * kMaxN * kMaxN;
    a.coef = coef;
    a.accumulate = accumulate;
    a.mode = mode;
    const int G = grid_size();
    int wpb = kApplyThreads / 32;
    bool big = false;
    for (int k = 0; k < L.D; ++k) big = big || L.n[k] > kMaxNTile;
    if (big) {   // a mode longer than the tiled passes take
        a.keys = s.keys;
        k_pass_point<R><<<G * 8, 256, 0, st>>>(a);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    }
    if (sizeof(R) == 4 && L.n[mode] <= kTcMaxN && L.nlast <= kTcMaxN)   // FP32: tensor cores
        return tc_pass(s, (const float2*)in, (float2*)out, (const float*)a.mat, mode, coef, accumulate,
                       in_scale, a.skip, a.skip_k, st);
    if (mode == L.D - 1) {
        const int nl = L.nlast;
        const size_t sm = (size_t)((nl * nl + 1) & ~1) * esz + (size_t)wpb * kMaxNTile * 2 * esz;
        a.wpb = wpb;
        a.units = s.rows;
        a.units_cap = s.rows_cap;
        a.nunits = s.cnt + CNT_ROWS;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass_row<R>, kApplyThreads, sm);
        k_pass_row<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    }
    const int nk = L.n[mode], nl = L.nlast;
    auto smem = [&](int wp) {
        return (size_t)wp * ((size_t)nk * nl * 2 * esz + kMaxNTile * 12) + (size_t)nk * nk * esz;
    };
    while (wpb > 1 && smem(wpb) > kSmemBudget) --wpb;
    a.wpb = wpb;
    a.units = s.leaders + (size_t)mode * s.rows_cap;
    a.units_cap = s.rows_cap;
    a.nunits = s.cnt + CNT_LEAD0 + mode;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass_fibre<R>, kApplyThreads, smem(wpb));
    k_pass_fibre<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, smem(wpb), st>>>(a);
    PQ_CHECK_LAUNCH();
    return PQ_OK;
}

// H.in for a generic SoP: merged single-mode matrices (one pass per mode),
// then every multi-factor term through the scratch vectors, last mode first.
template <typename R>
static pq_status launch_generic(const State& s, ApplyArgs<R> a, const void* in, void* out,
                                const double* in_scale, cudaStream_t st) {
    const Lattice& L = s.lat;
    static bool attr[2] = {false, false};
    const int pi = sizeof(R) == 8 ? 1 : 0;
    if (!attr[pi]) {
        PQ_CUDA_TRY(cudaFuncSetAttribute(k_pass_fibre<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        PQ_CUDA_TRY(cudaFuncSetAttribute(k_pass_row<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        attr[pi] = true;
    }
    bool first = true;
    pq_status rc;
    for (int k = L.D - 1; k >= 0; --k) {
        if (s.gsingle[k] < 0) continue;
        if ((rc = launch_pass<R>(s, a, k, s.gsingle[k], in, out, in_scale, 1.0, first ? 0 : 1, st)))
            return rc;
        first = false;
    }
    if (first) {
        k_zero<R><<<grid_size() * 4, 256, 0, st>>>((typename Cx<R>::T*)out, s.cnt + CNT_NA, a.skip,
                                                   a.skip_k);
        PQ_CHECK_LAUNCH();
    }
    const size_t esz = 2 * sizeof(R);
    for (const State::GPlan& plan : s.gplan) {
        const void* cur = in;
        const double* sc = in_scale;
        int tsel = 0;
        for (size_t p = 0; p < plan.passes.size(); ++p) {
            const bool last = p + 1 == plan.passes.size();
            void* dst = last ? out : (void*)((char*)s.gtmp + (size_t)tsel * s.cap * esz);
            if ((rc = launch_pass<R>(s, a, plan.passes[p].mode, plan.passes[p].mat, cur, dst, sc,
                                     last ? plan.coef : 1.0, last ? 1 : 0, st)))
                return rc;
            cur = dst;
            sc = nullptr;
            tsel ^= 1;
        }
    }
    return PQ_OK;
}

// ------------------------------------------------------------------------
// Element-parallel fibre kernels (n[k] <= 32, n[D-1] <= 32), the FP64 path.
// One warp per fibre (or plane): the warp compacts the fibre's active rows
// with a ballot, the lanes gather the fibre's active coefficients (lane e takes
// elements e, e + 32, ..., located by a monotone walk over the row offsets)
// into a zero-filled shared-memory tile, and each lane then forms the outputs
// of its elements over the fibre's active rows (and, in the inner pass, over
// the row's span and the potential).  Every output costs one FMA pair per
// active term, the fewest FP64 operations of the tiled kernels, which is what
// counts at GB300's FP64 rate; the FP32 path uses the item-blocked kernels
// below.

constexpr int kEpBatch = 8;          // warps per CTA, one fibre each

// position of the n-th (0-based) set bit of b
__device__ __forceinline__ int nth_set_bit(uint32_t b, int n) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const uint32_t lo = b & ((1u << w) - 1u);
        const int c = __popc(lo);
        if (n >= c) {
            n -= c;
            b >>= w;
            pos += w;
        } else {
            b = lo;
        }
    }
    return pos;
}

struct EpMeta {
    int na[kEpBatch];
    int eoff[kEpBatch + 1];
    uint32_t rst[kEpBatch][32];
    uint32_t rbt[kEpBatch][32];
    int rj[kEpBatch][32];
    int roff[kEpBatch][33];
};

// Phase 1 for warp f: compact the active rows (given per lane j < n) and
// their element offsets.
__device__ __forceinline__ void ep_compact(EpMeta& m, int f, int lane, int j, uint32_t b,
                                           uint32_t st) {
    const unsigned act = __ballot_sync(0xffffffffu, b != 0);
    const int slot = __popc(act & ((1u << lane) - 1u));
    const int cnt = b ? __popc(b) : 0;
    int x = cnt;   // inclusive scan of element counts over lanes (slot order = lane order)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (b) {
        m.rst[f][slot] = st;
        m.rbt[f][slot] = b;
        m.rj[f][slot] = j;
        m.roff[f][slot] = x - cnt;
    }
    const int total = __shfl_sync(0xffffffffu, x, 31);
    if (lane == 0) {
        m.na[f] = __popc(act);
        m.roff[f][__popc(act)] = total;
    }
}

// Element e of the warp's fibre, located from the lane's previous row:
// lanes walk their elements in increasing order, so the row index only moves
// forward (amortised O(1) instead of a binary search).
__device__ __forceinline__ void ep_next(const EpMeta& m, int f, int e, int& u, int& s,
                                        uint32_t& pos) {
    while (m.roff[f][u + 1] <= e) ++u;
    const int kth = e - m.roff[f][u];
    s = nth_set_bit(m.rbt[f][u], kth);
    pos = m.rst[f][u] + (uint32_t)kth;
}

// One warp per fibre; lanes work over the fibre's active coefficients.
template <typename R>
__global__ void __launch_bounds__(kApplyThreads) k_outer_ep(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int k = a.mode, nk = L.n[k], nl = L.nlast;
    const uint32_t rs = L.rstride[k];
    __shared__ EpMeta m;
    V* tiles = reinterpret_cast<V*>(smem);                           // [kEpBatch][nk][nl]
    R* Tk = reinterpret_cast<R*>(tiles + (size_t)kEpBatch * nk * nl);  // [nk][nk]
    for (int i = threadIdx.x; i < nk * nk; i += blockDim.x)
        Tk[i] = a.T[(size_t)k * kMaxN * kMaxN + (i / nk) * kMaxN + (i % nk)];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    V* tile = tiles + (size_t)w * nk * nl;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
    for (int64_t u = (int64_t)blockIdx.x * kEpBatch + w; u < nunits;
         u += (int64_t)gridDim.x * kEpBatch) {
        const uint32_t r0 = a.units[u];
        const int i0 = (int)((r0 / rs) % (uint32_t)nk);
        uint32_t b = 0, st = 0;
        if (lane < nk && lane >= i0) {
            const uint32_t r = r0 + (uint32_t)(lane - i0) * rs;
            if (a.rowinfo) {
                const uint2 ri = a.rowinfo[r];
                st = ri.x;
                b = ri.y;
            } else {
                b = (uint32_t)row_bits(a.bits, r, nl);
                if (b) st = rank_of(a.bits, a.off, (uint64_t)r * nl);
            }
        }
        ep_compact(m, w, lane, lane, b, st);
        __syncwarp();
        const int na = m.na[w], E = m.roff[w][na];
        for (int i = lane; i < na * nl; i += 32) tile[i] = cmake<R>(0, 0);
        __syncwarp();
        int row = 0;
        for (int e = lane; e < E; e += 32) {            // gather
            int sc;
            uint32_t pos;
            ep_next(m, w, e, row, sc, pos);
            V x = a.in[pos];
            x.x *= scale;
            x.y *= scale;
            tile[row * nl + sc] = x;
        }
        __syncwarp();
        row = 0;
#pragma unroll 1
        for (int e = lane; e < E; e += 32) {            // dot products, accumulate
            int sc;
            uint32_t pos;
            ep_next(m, w, e, row, sc, pos);
            V* o = a.out + pos;
            V ov = *o;
            const R* tj = Tk + m.rj[w][row] * nk;
            R ax = 0, ay = 0;
            for (int v = 0; v < na; ++v) {
                const R t = tj[m.rj[w][v]];
                const V cv = tile[v * nl + sc];
                ax += t * cv.x;
                ay += t * cv.y;
            }
            ov.x += ax;
            ov.y += ay;
            *o = ov;
        }
        __syncwarp();
    }
}

template <typename R>
static size_t smem_outer_ep(int nk, int nl) {
    return (size_t)kEpBatch * nk * nl * 2 * sizeof(R) + (size_t)nk * nk * sizeof(R);
}

// Inner pass, one warp per plane, lanes over the plane's active coefficients:
// mode D-2 over the plane's active rows, mode D-1 over the row's active span,
// the potential split as in k_apply_inner_reg (f(j) + g(s) + both-mode terms).
template <typename R>
__device__ __forceinline__ typename Cx<R>::T inner_ep_value(
    const ApplyArgs<R>& a, const EpMeta& m, int w, const typename Cx<R>::T* tile, const R* Tq,
    const R* Tlt, const R* pref, const R* fj, const R* gs, int n2, int nl, int D, int g3, int nt,
    int uu, int sc) {
    using V = typename Cx<R>::T;
    const int na = m.na[w];
    const int j = m.rj[w][uu];
    const R* tc = Tq + uu * n2;                         // compact T^(D-2) row of uu
    R ax = 0, ay = 0;
    for (int v = 0; v < na; ++v) {                      // mode D-2
        const R t = tc[v];
        const V c = tile[v * nl + sc];
        ax += t * c.x;
        ay += t * c.y;
    }
    const uint32_t rb = m.rbt[w][uu];                   // mode D-1 over the row's span
    const int slo = __ffs(rb) - 1, shi = 31 - __clz(rb);
    const V* row = tile + uu * nl;
    for (int ss = slo; ss <= shi; ++ss) {
        const R t = Tlt[ss * nl + sc];
        const V c = row[ss];
        ax += t * c.x;
        ay += t * c.y;
    }
    R vv = fj[uu] + gs[sc];
    for (int t = g3; t < nt; ++t)
        vv += pref[t] * a.pot[((size_t)t * D + D - 2) * kMaxN + j] *
              a.pot[((size_t)t * D + D - 1) * kMaxN + sc];
    const V c = row[sc];
    ax += vv * c.x;
    ay += vv * c.y;
    return cmake<R>(ax, ay);
}

template <typename R>
__global__ void __launch_bounds__(kApplyThreads) k_inner_ep(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int D = L.D, n2 = L.n[D - 2], nl = L.nlast, nt = a.nterms;
    const int g1 = a.ngroup[0], g2 = g1 + a.ngroup[1], g3 = g2 + a.ngroup[2];
    __shared__ EpMeta m;
    V* tiles = reinterpret_cast<V*>(smem);                             // [kEpBatch][n2][nl]
    R* prefs = reinterpret_cast<R*>(tiles + (size_t)kEpBatch * n2 * nl); // [kEpBatch][kMaxTerms]
    R* fjs = prefs + (size_t)kEpBatch * kMaxTerms;                       // [kEpBatch][32]
    R* gss = fjs + (size_t)kEpBatch * 32;                                // [kEpBatch][32]
    R* Tq = gss + (size_t)kEpBatch * 32;                                 // [n2][n2]
    R* Tlt = Tq + n2 * n2;                                               // [nl][nl]: Tlt[ss][s] = T[s][ss]
    R* Tcs = Tlt + nl * nl;                                              // [kEpBatch][n2][n2] compact T^(D-2)
    for (int i = threadIdx.x; i < n2 * n2; i += blockDim.x)
        Tq[i] = a.T[(size_t)(D - 2) * kMaxN * kMaxN + (i / n2) * kMaxN + (i % n2)];
    for (int i = threadIdx.x; i < nl * nl; i += blockDim.x)
        Tlt[i] = a.T[(size_t)(D - 1) * kMaxN * kMaxN + (i % nl) * kMaxN + (i / nl)];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    V* tile = tiles + (size_t)w * n2 * nl;
    R* Tc = Tcs + (size_t)w * n2 * n2;
    R* pref = prefs + (size_t)w * kMaxTerms;
    R* fj = fjs + (size_t)w * 32;
    R* gs = gss + (size_t)w * 32;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
    for (int64_t u = (int64_t)blockIdx.x * kEpBatch + w; u < nunits;
         u += (int64_t)gridDim.x * kEpBatch) {
        const uint32_t P = a.units[u];
        uint32_t b = 0, st = 0;
        if (lane < n2) {
            const uint32_t r = P * (uint32_t)n2 + (uint32_t)lane;
            if (a.rowinfo) {
                const uint2 ri = a.rowinfo[r];
                st = ri.x;
                b = ri.y;
            } else {
                b = (uint32_t)row_bits(a.bits, r, nl);
                if (b) st = rank_of(a.bits, a.off, (uint64_t)r * nl);
            }
        }
        ep_compact(m, w, lane, lane, b, st);
        for (int t = lane; t < nt; t += 32) {
            R p = a.potc[t];
            for (int kk = 0; kk < D - 2; ++kk) {
                const int d = (int)((P / L.pstride[kk]) % (uint32_t)L.n[kk]);
                p *= a.pot[((size_t)t * D + kk) * kMaxN + d];
            }
            pref[t] = p;
        }
        __syncwarp();
        const int na = m.na[w], E = m.roff[w][na];
        if (lane < na) {   // f(j) of compact row `lane`
            const int j = m.rj[w][lane];
            R f = 0;
            for (int t = 0; t < g1; ++t) f += pref[t];
            for (int t = g1; t < g2; ++t) f += pref[t] * a.pot[((size_t)t * D + D - 2) * kMaxN + j];
            fj[lane] = f;
        }
        if (lane < nl) {   // g(s)
            R g = 0;
            for (int t = g2; t < g3; ++t) g += pref[t] * a.pot[((size_t)t * D + D - 1) * kMaxN + lane];
            gs[lane] = g;
        }
        for (int i = lane; i < na * nl; i += 32) tile[i] = cmake<R>(0, 0);
        if (lane < na) {   // compact operator: Tc[uu][v] = T^(D-2)[j_uu][j_v], lane = v
            const int jv = m.rj[w][lane];
            for (int uu = 0; uu < na; ++uu) Tc[uu * n2 + lane] = Tq[m.rj[w][uu] * n2 + jv];
        }
        __syncwarp();
        int row = 0;
        for (int e = lane; e < E; e += 32) {            // gather
            int sc;
            uint32_t pos;
            ep_next(m, w, e, row, sc, pos);
            V x = a.in[pos];
            x.x *= scale;
            x.y *= scale;
            tile[row * nl + sc] = x;
        }
        __syncwarp();
        row = 0;
#pragma unroll 1
        for (int e = lane; e < E; e += 32) {            // outputs
            int sc;
            uint32_t pos;
            ep_next(m, w, e, row, sc, pos);
            a.out[pos] = inner_ep_value<R>(a, m, w, tile, Tc, Tlt, pref, fj, gs, n2, nl, D, g3, nt,
                                           row, sc);
        }
        __syncwarp();
    }
}

template <typename R>
static size_t smem_inner_ep(int n2, int nl) {
    return (size_t)kEpBatch * n2 * nl * 2 * sizeof(R) +
           ((size_t)kEpBatch * (kMaxTerms + 64 + n2 * n2) + n2 * n2 + nl * nl) * sizeof(R);
}

// ------------------------------------------------------------------------
// Item-blocked fibre kernels (n[k] <= 32, n[D-1] <= 32), the FP32 fast path.
// One warp per fibre (outer) or plane (inner).  The fibre's active rows are
// compacted with a ballot; each lane then owns (row, item) work units, an item
// being W consecutive last-mode points.  Gather: every item of every active
// row is staged in shared memory (zeros where inactive), the non-empty items
// going to a per-warp list.  Compute: a lane forms the W outputs of its item
// together, so each operator element and each staged input is loaded once per
// W outputs with 16-byte shared-memory loads; positions come from the row's
// start and one popcount.  The rows of a fibre are contiguous ranges
// of A, so the global loads and stores of an item touch consecutive addresses.

constexpr int kQWarps = kApplyThreads / 32;
// Last-mode points per work item (build-time; 4, 6 or 8), for the inner and
// the outer passes.  On the 6D 24^6 ellipsoid (9.97e6 points) one H.psi took
// 749 us with 4 / 4, 717 us with 6 / 6 and 1082 us with 8 / 8; under ncu the
// inner pass ran 213 us with 4 and 231 us with 6 (its larger code waits for
// instructions), the outer passes 131 us with 4 and 119 us with 6.
#ifndef PQ_QW_INNER
#define PQ_QW_INNER 4
#endif
#ifndef PQ_QW_OUTER
#define PQ_QW_OUTER 6
#endif
constexpr int kQWInner = PQ_QW_INNER;
constexpr int kQWOuter = PQ_QW_OUTER;

struct __align__(16) QuadMeta {   // per warp, per fibre
    uint32_t rst[32];           // first position in A of compact row u
    uint32_t rbt[32];           // last-mode pattern of compact row u
    int rj[32];                 // fibre index of compact row u
    uint16_t item[32 * 8];      // (u << 3) | q of the non-empty items
};

// W consecutive complex values (16-byte aligned: W even for float, any W for double)
template <typename R, int W>
__device__ __forceinline__ void ld_w(const typename Cx<R>::T* p, typename Cx<R>::T (&x)[W]) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {
            const float4 v = reinterpret_cast<const float4*>(p)[h];
            x[2 * h] = make_float2(v.x, v.y);
            x[2 * h + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int t = 0; t < W; ++t) x[t] = p[t];
    }
}

template <typename R, int W>
__device__ __forceinline__ void st_w(typename Cx<R>::T* p, const typename Cx<R>::T (&x)[W]) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int h = 0; h < W / 2; ++h)
            reinterpret_cast<float4*>(p)[h] =
                make_float4(x[2 * h].x, x[2 * h].y, x[2 * h + 1].x, x[2 * h + 1].y);
    } else {
#pragma unroll
        for (int t = 0; t < W; ++t) p[t] = x[t];
    }
}

// W consecutive real values (8-byte aligned for float, W even)
template <typename R, int W>
__device__ __forceinline__ void ld_real_w(const R* p, R (&t)[W]) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {
            const float2 v = reinterpret_cast<const float2*>(p)[h];
            t[2 * h] = v.x;
            t[2 * h + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int h = 0; h < W; ++h) t[h] = p[h];
    }
}

// Row table entry of lattice row r: first position in A and pattern.
template <typename R>
__device__ __forceinline__ void q_row(const ApplyArgs<R>& a, uint32_t r, int nl, uint32_t& b,
                                      uint32_t& st) {
    if (a.rowinfo) {
        const uint2 ri = a.rowinfo[r];
        st = ri.x;
        b = ri.y;
    } else {
        b = (uint32_t)row_bits(a.bits, r, nl);
        st = b ? rank_of(a.bits, a.off, (uint64_t)r * nl) : 0u;
    }
}

// Compact the fibre's active rows (lane j holds row j's pattern b and start
// st) into m; returns the number of active rows.
__device__ __forceinline__ int q_compact(QuadMeta& m, int lane, uint32_t b, uint32_t st) {
    const unsigned act = __ballot_sync(0xffffffffu, b != 0);
    if (b) {
        const int slot = __popc(act & ((1u << lane) - 1u));
        m.rst[slot] = st;
        m.rbt[slot] = b;
        m.rj[slot] = lane;
    }
    return __popc(act);
}

// Stage all W-point items of the na active rows into tile (row stride nlw,
// zeros where inactive) and list the non-empty ones in m.item; returns the
// number of items.  Lane owns row offset gu and item column gq of each round
// of rpr rows.
template <typename R, int W>
__device__ __forceinline__ int q_gather(const ApplyArgs<R>& a, QuadMeta& m, typename Cx<R>::T* tile,
                                        int na, int nlw, int rpr, int gu, int gq, int lane,
                                        R scale, uint64_t nact) {
    using V = typename Cx<R>::T;
    constexpr uint32_t kMask = (1u << W) - 1u;
    int nitems = 0;
    for (int u0 = 0; u0 < na; u0 += rpr) {
        const int uu = u0 + gu;
        uint32_t bq = 0;
        if (gu < rpr && uu < na) {
            const uint32_t rb = m.rbt[uu];
            bq = (rb >> (W * gq)) & kMask;
            uint32_t pos = m.rst[uu] + (uint32_t)__popc(rb & ((1u << (W * gq)) - 1u));
            V x[W];
#pragma unroll
            for (int t = 0; t < W; ++t) {
                x[t] = cmake<R>(0, 0);
                if ((bq >> t) & 1u) {
                    if (pq_in_bounds(pos, nact, 23, a.cnt)) {
                        x[t] = a.in[pos];
                        x[t].x *= scale;
                        x[t].y *= scale;
                    }
                    ++pos;
                }
            }
            st_w<R, W>(tile + uu * nlw + W * gq, x);
        }
        const unsigned ne = __ballot_sync(0xffffffffu, bq != 0);
        if (bq) m.item[nitems + __popc(ne & ((1u << lane) - 1u))] = (uint16_t)((uu << 3) | gq);
        nitems += __popc(ne);
    }
    return nitems;
}

// acc += t x for a real t and a complex x: one packed two-lane FMA in FP32
// (the same fused operation on each of re and im), two FMAs in FP64.
__device__ __forceinline__ void cfma(float2& acc, float t, float2 x) {
    acc = __ffma2_rn(make_float2(t, t), x, acc);
}
__device__ __forceinline__ void cfma(double2& acc, double t, double2 x) {
    acc.x = fma(t, x.x, acc.x);
    acc.y = fma(t, x.y, acc.y);
}

// acc[t] += sum_v trow[rj[v]] x[v][W q + t] over the compact rows.
template <typename R, int W>
__device__ __forceinline__ void q_column(const R* trow, const int* rj, const typename Cx<R>::T* xcol,
                                         int na, int nlw, typename Cx<R>::T (&acc)[W]) {
    using V = typename Cx<R>::T;
    for (int v = 0; v < na; ++v) {
        const R tv = trow[rj[v]];
        V x[W];
        ld_w<R, W>(xcol + v * nlw, x);
#pragma unroll
        for (int t = 0; t < W; ++t) cfma(acc[t], tv, x[t]);
    }
}

// out[p] += v.  Each output receives one contribution per pass (its one
// fibre), so the sum is the same as a load-add-store; the reduction at L2
// leaves nothing for the warp to wait on.
__device__ __forceinline__ void q_accumulate(float2* p, float2 v) { atomicAdd(p, v); }
__device__ __forceinline__ void q_accumulate(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

// Items per row for width W and last-mode length nl.
__host__ __device__ constexpr int q_items_per_row(int nl, int W) { return (nl + W - 1) / W; }

template <typename R, int W>
__global__ void __launch_bounds__(kApplyThreads) k_outer_q(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (gated_off(a)) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ QuadMeta meta[kQWarps];
    const Lattice& L = a.L;
    const int k = a.mode, nk = L.n[k], nl = L.nlast;
    const int nq = q_items_per_row(nl, W), nlw = nq * W, nkp = nk | 1;
    const uint32_t rs = L.rstride[k];
    V* tiles = reinterpret_cast<V*>(smem);                            // [kQWarps][nk][nlw]
    R* Tk = reinterpret_cast<R*>(tiles + (size_t)kQWarps * nk * nlw);   // [nk][nkp]
    for (int i = threadIdx.x; i < nk * nk; i += blockDim.x) {
        const int r = i / nk, c = i - r * nk;
        Tk[r * nkp + c] = a.T[(size_t)k * kMaxN * kMaxN + r * kMaxN + c];
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    QuadMeta& m = meta[w];
    V* tile = tiles + (size_t)w * nk * nlw;
    const int rpr = 32 / nq, gu = lane / nq, gq = lane - gu * nq;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
#ifdef PQ_BOUNDS_CHECK
    const uint64_t nact = (uint64_t)a.cnt[CNT_NA];
#else
    const uint64_t nact = 0;
#endif
    for (int64_t u = (int64_t)blockIdx.x * kQWarps + w; u < nunits;
         u += (int64_t)gridDim.x * kQWarps) {
        if (!pq_in_bounds((uint64_t)u, a.units_cap, 21, a.cnt)) break;
        const uint32_t r0 = a.units[u];
        if (!pq_in_bounds(r0, L.nrows, 22, a.cnt)) continue;
        const int i0 = (int)((r0 / rs) % (uint32_t)nk);
        uint32_t b = 0, st = 0;
        if (lane < nk && lane >= i0) q_row<R>(a, r0 + (uint32_t)(lane - i0) * rs, nl, b, st);
        const int na = q_compact(m, lane, b, st);
        __syncwarp();
        const int nitems = q_gather<R, W>(a, m, tile, na, nlw, rpr, gu, gq, lane, scale, nact);
        __syncwarp();
#pragma unroll 1
        for (int e = lane; e < nitems; e += 32) {
            const int it = m.item[e];
            const int uu = it >> 3, q = it & 7;
            const uint32_t rb = m.rbt[uu];
            const uint32_t bq = (rb >> (W * q)) & ((1u << W) - 1u);
            V acc[W];
#pragma unroll
            for (int t = 0; t < W; ++t) acc[t] = cmake<R>(0, 0);
            q_column<R, W>(Tk + m.rj[uu] * nkp, m.rj, tile + W * q, na, nlw, acc);
            uint32_t p = m.rst[uu] + (uint32_t)__popc(rb & ((1u << (W * q)) - 1u));
#pragma unroll
            for (int t = 0; t < W; ++t) {
                if ((bq >> t) & 1u) {
                    if (pq_in_bounds(p, nact, 25, a.cnt)) q_accumulate(a.out + p, acc[t]);
                    ++p;
                }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------
// Dense-tile passes (FP32), for sets that cover at least half the lattice
// (the 6D Henon-Heiles set fills the whole 24^6 lattice after about 100
// steps).  A block stages whole tiles of the lattice in shared memory, each
// point found through the row table (row start in A and pattern: position =
// start + popcount of the pattern below the point) and zero where inactive, and
// treats the tile as dense: the passes are batched contractions with no
// compaction or item lists, and only active outputs are written.  Each thread
// owns a 4 x 4 block of outputs (four fibre points by four last-mode points)
// in registers, so one 16-byte shared-memory load of operator entries and two
// of coefficients feed 16 packed complex FMAs.
//   inner pass: kDensePlanes planes (modes D-2 and D-1 with the other digits
//     fixed) per block; both modes and the SoP potential; each output written
//     once;
//   pair pass over outer modes (k, k+1): a tile of n[k] x n[k+1] rows (the
//     rows that differ only in digits k and k+1) by kDenseC last-mode points
//     per block; both modes, added to the output in place (the block owns
//     these outputs in this pass).
// Both run a two-stage pipeline over their units: the asynchronous copies of
// the next unit are in flight while the block computes the current one from
// the other buffer.  The products are linear in the input, so the Krylov
// scale is applied to the results.
constexpr int kDenseThreads = 288;
constexpr int kDensePlanes = 8;
constexpr int kDenseC = 8;

// acc[r][q] += t[r] x[q]
__device__ __forceinline__ void outer4(float2 (&acc)[4][4], const float4& t, const float2 (&x)[4]) {
    const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(acc[r][q], tv[r], x[q]);
}

__device__ __forceinline__ void ld4(const float2* p, float2 (&x)[4]) {
    const float4 u = reinterpret_cast<const float4*>(p)[0];
    const float4 v = reinterpret_cast<const float4*>(p)[1];
    x[0] = make_float2(u.x, u.y);
    x[1] = make_float2(u.z, u.w);
    x[2] = make_float2(v.x, v.y);
    x[3] = make_float2(v.z, v.w);
}

__device__ __forceinline__ void st4(float2* p, const float2 (&x)[4]) {
    reinterpret_cast<float4*>(p)[0] = make_float4(x[0].x, x[0].y, x[1].x, x[1].y);
    reinterpret_cast<float4*>(p)[1] = make_float4(x[2].x, x[2].y, x[3].x, x[3].y);
}

// 8-byte asynchronous global -> shared copy; zero-fills the destination when
// !valid (no bytes are read then).
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    const int nb = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gsrc), "r"(nb)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}

// Stage points [c0, c0 + n) of a lattice row with row-table entry ri at sdst
// (16-byte aligned, n even), zero where inactive: 16-byte copies when the span
// is fully active and its source address is 16-byte aligned, else one 8-byte
// copy (or zero fill) per point.
__device__ __forceinline__ void stage_row(float2* sdst, const float2* in, uint2 ri, int c0, int n) {
    const uint32_t full = n >= 32 ? ~0u : (1u << n) - 1u;
    const uint32_t m = (ri.y >> c0) & full;
    uint32_t pos = ri.x + (uint32_t)__popc(ri.y & ((1u << c0) - 1u));
    if (m == full && !(reinterpret_cast<uintptr_t>(in + pos) & 15u)) {
        for (int h = 0; h < n / 2; ++h) cp_async16(sdst + 2 * h, in + pos + 2 * h);
        return;
    }
    for (int c = 0; c < n; ++c) {
        const bool on = (m >> c) & 1u;
        cp_async8(sdst + c, on ? in + pos : in, on);
        pos += on ? 1u : 0u;
    }
}

// The dense-tile kernels keep three row-table buffers and two coefficient
// buffers: in the iteration of unit u the block copies the coefficients of
// the next unit (rows staged one iteration earlier) and the row-table entries
// of the unit after it, and computes u; one wait and one barrier per unit.

// Inner pass on a dense set: y = T^{D-2} x + T^{D-1} x + V x per plane.
__global__ void __launch_bounds__(kDenseThreads) k_dense_inner(ApplyArgs<float> a) {
    if (a.skip && *a.skip <= a.skip_k) return;
    if (gated_off(a)) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int D = L.D, n2 = L.n[D - 2], nl = L.nlast, nt = a.nterms, pl = n2 * nl;
    const int g1 = a.ngroup[0], g2 = g1 + a.ngroup[1], g3 = g2 + a.ngroup[2];
    float2* Xb = reinterpret_cast<float2*>(smem);                         // [2][P][n2][nl]
    float* T2 = reinterpret_cast<float*>(Xb + (size_t)2 * kDensePlanes * pl);   // [j][i] = T^{D-2}[i][j]
    float* Tl = T2 + n2 * n2;                                             // [s][c] = T^{D-1}[c][s]
    float* Vr = Tl + nl * nl;                                             // [P][n2] (with the constant)
    float* Vs = Vr + kDensePlanes * n2;                                   // [P][nl]
    float* pf = Vs + kDensePlanes * nl;                                   // [P][nt] term prefactors
    const int nboth = nt - g3;
    float* F2 = pf + kDensePlanes * (nt > 1 ? nt : 1);                   // [nboth][n2] both-mode factors
    float* F3 = F2 + nboth * n2;                                          // [nboth][nl]
    uint2* Rb = reinterpret_cast<uint2*>(((uintptr_t)(F3 + nboth * nl) + 15) & ~(uintptr_t)15);   // [3][P * n2]
    for (int i = threadIdx.x; i < nboth * n2; i += blockDim.x)
        F2[i] = a.pot[((size_t)(g3 + i / n2) * D + D - 2) * kMaxN + i % n2];
    for (int i = threadIdx.x; i < nboth * nl; i += blockDim.x)
        F3[i] = a.pot[((size_t)(g3 + i / nl) * D + D - 1) * kMaxN + i % nl];
    for (int i = threadIdx.x; i < n2 * n2; i += blockDim.x) {
        const int j = i / n2, r = i - j * n2;
        T2[i] = a.T[(size_t)(D - 2) * kMaxN * kMaxN + r * kMaxN + j];
    }
    for (int i = threadIdx.x; i < nl * nl; i += blockDim.x) {
        const int sp = i / nl, c = i - sp * nl;
        Tl[i] = a.T[(size_t)(D - 1) * kMaxN * kMaxN + c * kMaxN + sp];
    }
    const float scale = a.in_scale ? (float)(*a.in_scale) : 1.f;
    const int nab = n2 / 4, ncb = nl / 4;
    const uint32_t nunits = (L.nplanes + kDensePlanes - 1) / kDensePlanes;
    auto nplanes_of = [&](uint32_t u) {
        return (int)min((uint32_t)kDensePlanes, L.nplanes - u * kDensePlanes);
    };
    auto fetch_rows = [&](uint32_t u, int r3) {   // the unit's rows are consecutive
        const uint64_t r0 = (uint64_t)u * kDensePlanes * n2;
        uint2* dst = Rb + (size_t)r3 * kDensePlanes * n2;
        for (int i = threadIdx.x; i < nplanes_of(u) * n2; i += blockDim.x)
            cp_async8(dst + i, a.rowinfo + r0 + i, true);
    };
    auto issue = [&](uint32_t u, int buf, const uint2* R) {
        float2* dst = Xb + (size_t)buf * kDensePlanes * pl;
        for (int rowi = threadIdx.x; rowi < nplanes_of(u) * n2; rowi += blockDim.x)
            stage_row(dst + (size_t)rowi * nl, a.in, R[rowi], 0, nl);
    };
    const uint32_t G = gridDim.x;
    if (blockIdx.x < nunits) {
        fetch_rows(blockIdx.x, 0);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        issue(blockIdx.x, 0, Rb);
        if (blockIdx.x + G < nunits) fetch_rows(blockIdx.x + G, 1);
        cp_async_commit();
    }
    int it = 0;
    for (uint32_t u = blockIdx.x; u < nunits; u += G, ++it) {
        const uint32_t P0 = u * kDensePlanes;
        const int np = nplanes_of(u);
        cp_async_wait_all();
        __syncthreads();   // this unit's coefficients and the next unit's rows
        if (u + G < nunits) issue(u + G, (it + 1) & 1, Rb + (size_t)((it + 1) % 3) * kDensePlanes * n2);
        if (u + 2 * G < nunits) fetch_rows(u + 2 * G, (it + 2) % 3);
        cp_async_commit();
        const float2* X = Xb + (size_t)(it & 1) * kDensePlanes * pl;
        const uint2* R = Rb + (size_t)(it % 3) * kDensePlanes * n2;
        // term prefactors over the plane's other digits
        for (int i = threadIdx.x; i < np * nt; i += blockDim.x) {
            const int p = i / nt, t = i - p * nt;
            const uint32_t P = P0 + (uint32_t)p;
            float v = a.potc[t];
            for (int kk = 0; kk < D - 2; ++kk) {
                const int d = (int)((P / L.pstride[kk]) % (uint32_t)L.n[kk]);
                v *= a.pot[((size_t)t * D + kk) * kMaxN + d];
            }
            pf[p * nt + t] = v;
        }
        __syncthreads();   // pf
        for (int i = threadIdx.x; i < np * n2; i += blockDim.x) {
            const int p = i / n2, r = i - p * n2;
            float v = 0.f;
            for (int t = 0; t < g1; ++t) v += pf[p * nt + t];
            for (int t = g1; t < g2; ++t) v += pf[p * nt + t] * a.pot[((size_t)t * D + D - 2) * kMaxN + r];
            Vr[p * n2 + r] = v;
        }
        for (int i = threadIdx.x; i < np * nl; i += blockDim.x) {
            const int p = i / nl, c = i - p * nl;
            float v = 0.f;
            for (int t = g2; t < g3; ++t) v += pf[p * nt + t] * a.pot[((size_t)t * D + D - 1) * kMaxN + c];
            Vs[p * nl + c] = v;
        }
        __syncthreads();
        for (int task = threadIdx.x; task < np * nab * ncb; task += blockDim.x) {
            const int p = task / (nab * ncb), rem = task - p * nab * ncb;
            const int i0 = (rem / ncb) * 4, c0 = (rem % ncb) * 4;
            const float2* Xp = X + (size_t)p * pl;
            float2 acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = make_float2(0.f, 0.f);
            // mode D-2: acc[r][q] += T[i0+r][j] x[j][c0+q]
#pragma unroll 4
            for (int j = 0; j < n2; ++j) {
                const float4 t = *reinterpret_cast<const float4*>(T2 + j * n2 + i0);
                float2 x[4];
                ld4(Xp + j * nl + c0, x);
                outer4(acc, t, x);
            }
            // mode D-1: acc[r][q] += T[c0+q][s] x[i0+r][s]
#pragma unroll 4
            for (int sp = 0; sp < nl; ++sp) {
                const float4 t = *reinterpret_cast<const float4*>(Tl + sp * nl + c0);
                const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float2 x = Xp[(i0 + r) * nl + sp];
#pragma unroll
                    for (int q = 0; q < 4; ++q) cfma(acc[r][q], tv[q], x);
                }
            }
            // potential; active outputs only, 16-byte stores for four active
            // points at a 16-byte aligned address
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint2 ri = R[p * n2 + i0 + r];
                const uint32_t mk = (ri.y >> c0) & 0xFu;
                float2 x[4];
                ld4(Xp + (i0 + r) * nl + c0, x);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v = Vr[p * n2 + i0 + r] + Vs[p * nl + c0 + q];
                    for (int t = 0; t < nboth; ++t)
                        v += pf[p * nt + g3 + t] * F2[t * n2 + i0 + r] * F3[t * nl + c0 + q];
                    cfma(acc[r][q], v, x[q]);
                    acc[r][q].x *= scale;
                    acc[r][q].y *= scale;
                }
                uint32_t pos = ri.x + (uint32_t)__popc(ri.y & ((1u << c0) - 1u));
                if (mk == 0xFu && !(reinterpret_cast<uintptr_t>(a.out + pos) & 15u)) {
                    st4(a.out + pos, acc[r]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if ((mk >> q) & 1u) a.out[pos++] = acc[r][q];
                }
            }
        }
        __syncthreads();   // X, pf and the tables are free for the next units
    }
}

// Pair pass on a dense set over outer modes (k, k+1): y += T^k x + T^{k+1} x.
__global__ void __launch_bounds__(kDenseThreads) k_dense_pair(ApplyArgs<float> a) {
    if (a.skip && *a.skip <= a.skip_k) return;
    if (gated_off(a)) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice& L = a.L;
    const int k = a.mode, na = L.n[k], nb = L.n[k + 1], nl = L.nlast, nbp = nb | 1;
    const uint32_t sa = L.rstride[k], sb = L.rstride[k + 1];
    const size_t tile = (size_t)na * nb * kDenseC;
    float2* Xb = reinterpret_cast<float2*>(smem);                         // [2][na][nb][kDenseC]
    float* Ta = reinterpret_cast<float*>(Xb + 2 * tile);                  // [j][a] = T^k[a][j]
    float* Tb = Ta + na * na;                                             // [b][j], row stride nbp
    uint2* Rb = reinterpret_cast<uint2*>(((uintptr_t)(Tb + nb * nbp) + 15) & ~(uintptr_t)15);   // [3][na * nb]
    for (int i = threadIdx.x; i < na * na; i += blockDim.x) {
        const int j = i / na, r = i - j * na;
        Ta[i] = a.T[(size_t)k * kMaxN * kMaxN + r * kMaxN + j];
    }
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
        const int r = i / nb, j = i - r * nb;
        Tb[r * nbp + j] = a.T[(size_t)(k + 1) * kMaxN * kMaxN + r * kMaxN + j];
    }
    const float scale = a.in_scale ? (float)(*a.in_scale) : 1.f;
    const int nch = nl / kDenseC, nab = na / 4, nab_rows = na * nb;
    const uint32_t ntiles = L.nrows / (uint32_t)(na * nb);
    const uint64_t nunits = (uint64_t)ntiles * nch;
    // row (t, 0, 0) and the first last-mode point of the unit's chunk
    auto unit_base = [&](uint64_t u, int& c0) -> uint64_t {
        const uint32_t t = (uint32_t)(u / nch);
        c0 = (int)(u - (uint64_t)t * nch) * kDenseC;
        const uint32_t hi = t / sb, lo = t - hi * sb;
        return (uint64_t)hi * sa * na + lo;
    };
    auto fetch_rows = [&](uint64_t u, int r3) {
        int c0;
        const uint64_t rbase = unit_base(u, c0);
        uint2* dst = Rb + (size_t)r3 * nab_rows;
        for (int rowi = threadIdx.x; rowi < nab_rows; rowi += blockDim.x) {
            const int ra = rowi / nb, rb = rowi - ra * nb;
            cp_async8(dst + rowi, a.rowinfo + rbase + (uint64_t)ra * sa + (uint64_t)rb * sb, true);
        }
    };
    auto issue = [&](uint64_t u, int buf, const uint2* R) {
        int c0;
        unit_base(u, c0);
        float2* dst = Xb + (size_t)buf * tile;
        for (int rowi = threadIdx.x; rowi < nab_rows; rowi += blockDim.x)
            stage_row(dst + (size_t)rowi * kDenseC, a.in, R[rowi], c0, kDenseC);
    };
    const uint64_t G = gridDim.x;
    if (blockIdx.x < nunits) {
        fetch_rows(blockIdx.x, 0);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();   // also the operator tables
        issue(blockIdx.x, 0, Rb);
        if (blockIdx.x + G < nunits) fetch_rows(blockIdx.x + G, 1);
        cp_async_commit();
    }
    int it = 0;
    for (uint64_t u = blockIdx.x; u < nunits; u += G, ++it) {
        cp_async_wait_all();
        __syncthreads();   // this unit's coefficients and the next unit's rows
        if (u + G < nunits) issue(u + G, (it + 1) & 1, Rb + (size_t)((it + 1) % 3) * nab_rows);
        if (u + 2 * G < nunits) fetch_rows(u + 2 * G, (it + 2) % 3);
        cp_async_commit();
        const uint2* R = Rb + (size_t)(it % 3) * nab_rows;
        const float2* X = Xb + (size_t)(it & 1) * tile;
        int c0;
        unit_base(u, c0);
        for (int task = threadIdx.x; task < nab * nb * (kDenseC / 4); task += blockDim.x) {
            const int cb = task % (kDenseC / 4), rem = task / (kDenseC / 4);
            const int rb = rem % nb, a0 = (rem / nb) * 4, cq = cb * 4;
            float2 acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = make_float2(0.f, 0.f);
            // mode k: acc[r][q] += T^k[a0+r][j] x[j][rb][cq+q]
#pragma unroll 4
            for (int j = 0; j < na; ++j) {
                const float4 tv = *reinterpret_cast<const float4*>(Ta + j * na + a0);
                float2 x[4];
                ld4(X + ((size_t)j * nb + rb) * kDenseC + cq, x);
                outer4(acc, tv, x);
            }
            // mode k+1: acc[r][q] += T^{k+1}[rb][j] x[a0+r][j][cq+q]
            const float* tb = Tb + rb * nbp;
#pragma unroll 2
            for (int j = 0; j < nb; ++j) {
                const float tv = tb[j];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float2 x[4];
                    ld4(X + ((size_t)(a0 + r) * nb + j) * kDenseC + cq, x);
#pragma unroll
                    for (int q = 0; q < 4; ++q) cfma(acc[r][q], tv, x[q]);
                }
            }
            // y += scale acc on the active points, two rows at a time with both
            // rows' loads before their stores (the positions are distinct);
            // 16-byte accesses for four active points at a 16-byte aligned
            // address
            const int cc = c0 + cq;
#pragma unroll
            for (int r0 = 0; r0 < 4; r0 += 2) {
                uint32_t pos0[2], mk[2];
                float2 y[2][4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint2 ri = R[(a0 + r0 + h) * nb + rb];
                    mk[h] = (ri.y >> cc) & 0xFu;
                    pos0[h] = ri.x + (uint32_t)__popc(ri.y & ((1u << cc) - 1u));
                    if (mk[h] == 0xFu && !(reinterpret_cast<uintptr_t>(a.out + pos0[h]) & 15u)) {
                        ld4(a.out + pos0[h], y[h]);
                    } else {
                        uint32_t pp = pos0[h];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if ((mk[h] >> q) & 1u) y[h][q] = a.out[pp++];
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        y[h][q].x = fmaf(scale, acc[r0 + h][q].x, y[h][q].x);
                        y[h][q].y = fmaf(scale, acc[r0 + h][q].y, y[h][q].y);
                    }
                    if (mk[h] == 0xFu && !(reinterpret_cast<uintptr_t>(a.out + pos0[h]) & 15u)) {
                        st4(a.out + pos0[h], y[h]);
                    } else {
                        uint32_t pp = pos0[h];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if ((mk[h] >> q) & 1u) a.out[pp++] = y[h][q];
                    }
                }
            }
        }
        __syncthreads();   // the buffer is refilled two units on
    }
}

static size_t smem_dense_inner(const Lattice& L, int nterms) {
    const int n2 = L.n[L.D - 2], nl = L.nlast;
    return (size_t)2 * kDensePlanes * n2 * nl * 8 + (size_t)(n2 * n2 + nl * nl) * 4 +
           (size_t)kDensePlanes * (n2 + nl + std::max(nterms, 1)) * 4 + (size_t)nterms * (n2 + nl) * 4 +
           16 + (size_t)3 * kDensePlanes * n2 * 8;
}

static size_t smem_dense_pair(const Lattice& L, int k) {
    const int na = L.n[k], nb = L.n[k + 1];
    return (size_t)2 * na * nb * kDenseC * 8 + (size_t)(na * na + nb * (nb | 1)) * 4 + 16 +
           (size_t)3 * na * nb * 8;
}

// The dense-tile passes take modes of at most 32 points (the row table holds
// 32-bit patterns), with n[D-2] and the pair modes' first mode multiples of 4
// and n[D-1] a multiple of kDenseC.
static bool dense_ok(const Lattice& L, int nterms) {
    if (L.D < 2 || L.nlast > 32 || L.nlast % kDenseC || L.n[L.D - 2] % 4 || L.n[L.D - 2] > 32)
        return false;
    return smem_dense_inner(L, nterms) <= kSmemBudget;
}

template <typename R, int W>
static size_t smem_outer_q(int nk, int nl) {
    const int nlw = q_items_per_row(nl, W) * W;
    return (size_t)kQWarps * nk * nlw * 2 * sizeof(R) + (size_t)nk * (nk | 1) * sizeof(R);
}

// Inner pass: modes D-2 (across the plane's active rows) and D-1 (along the
// row's active span) plus the SoP potential, split by the tile modes a term
// touches: f(j) (neither or D-2 only), g(s) (D-1 only), both-mode terms.
template <typename R, int W>
__global__ void __launch_bounds__(kApplyThreads) k_inner_q(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (gated_off(a)) return;
    if (a.cnt[CNT_ERR] & 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ QuadMeta meta[kQWarps];
    __shared__ R prefs[kQWarps][kMaxTerms];
    __shared__ R fjs[kQWarps][32];
    __shared__ __align__(16) R gss[kQWarps][40];   // nlw <= 36 for W = 6
    const Lattice& L = a.L;
    const int D = L.D, n2 = L.n[D - 2], nl = L.nlast, nt = a.nterms;
    const int nq = q_items_per_row(nl, W), nlw = nq * W, n2p = n2 | 1;
    const int g1 = a.ngroup[0], g2 = g1 + a.ngroup[1], g3 = g2 + a.ngroup[2];
    V* tiles = reinterpret_cast<V*>(smem);                             // [kQWarps][n2][nlw]
    R* Tlq = reinterpret_cast<R*>(tiles + (size_t)kQWarps * n2 * nlw);   // [nl][nlw]: T[s][s'] at [s'][s]
    R* potl = Tlq + (size_t)nl * nlw;                                    // [nt - g3][nlw]
    R* Tq = potl + (size_t)(nt - g3) * nlw;                              // [n2][n2p]
    for (int i = threadIdx.x; i < nl * nlw; i += blockDim.x) {
        const int sp = i / nlw, s = i - sp * nlw;
        Tlq[i] = s < nl ? a.T[(size_t)(D - 1) * kMaxN * kMaxN + s * kMaxN + sp] : (R)0;
    }
    for (int i = threadIdx.x; i < (nt - g3) * nlw; i += blockDim.x) {
        const int t = g3 + i / nlw, s = i % nlw;
        potl[i] = s < nl ? a.pot[((size_t)t * D + D - 1) * kMaxN + s] : (R)0;
    }
    for (int i = threadIdx.x; i < n2 * n2; i += blockDim.x) {
        const int r = i / n2, c = i - r * n2;
        Tq[r * n2p + c] = a.T[(size_t)(D - 2) * kMaxN * kMaxN + r * kMaxN + c];
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    QuadMeta& m = meta[w];
    V* tile = tiles + (size_t)w * n2 * nlw;
    R* pref = prefs[w];
    R* fj = fjs[w];
    R* gs = gss[w];
    const int rpr = 32 / nq, gu = lane / nq, gq = lane - gu * nq;
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    const int64_t nunits = *a.nunits;
#ifdef PQ_BOUNDS_CHECK
    const uint64_t nact = (uint64_t)a.cnt[CNT_NA];
#else
    const uint64_t nact = 0;
#endif
    for (int64_t u = (int64_t)blockIdx.x * kQWarps + w; u < nunits;
         u += (int64_t)gridDim.x * kQWarps) {
        if (!pq_in_bounds((uint64_t)u, a.units_cap, 26, a.cnt)) break;
        const uint32_t P = a.units[u];
        if (!pq_in_bounds(P, L.nplanes, 27, a.cnt)) continue;
        uint32_t b = 0, st = 0;
        if (lane < n2) q_row<R>(a, P * (uint32_t)n2 + (uint32_t)lane, nl, b, st);
        const int na = q_compact(m, lane, b, st);
        for (int t = lane; t < nt; t += 32) {
            R pv = a.potc[t];
            for (int kk = 0; kk < D - 2; ++kk) {
                const int d = (int)((P / L.pstride[kk]) % (uint32_t)L.n[kk]);
                pv *= a.pot[((size_t)t * D + kk) * kMaxN + d];
            }
            pref[t] = pv;
        }
        __syncwarp();
        if (lane < na) {   // f(j) of compact row `lane`
            const int j = m.rj[lane];
            R f = 0;
            for (int t = 0; t < g1; ++t) f += pref[t];
            for (int t = g1; t < g2; ++t) f += pref[t] * a.pot[((size_t)t * D + D - 2) * kMaxN + j];
            fj[lane] = f;
        }
        {   // g(s), zero in the padding
            R g = 0;
            if (lane < nl)
                for (int t = g2; t < g3; ++t)
                    g += pref[t] * a.pot[((size_t)t * D + D - 1) * kMaxN + lane];
            gs[lane] = g;
            if (lane < 8) gs[32 + lane] = 0;
        }
        const int nitems = q_gather<R, W>(a, m, tile, na, nlw, rpr, gu, gq, lane, scale, nact);
        __syncwarp();
#pragma unroll 1
        for (int e = lane; e < nitems; e += 32) {
            const int it = m.item[e];
            const int uu = it >> 3, q = it & 7;
            const uint32_t rb = m.rbt[uu];
            const uint32_t bq = (rb >> (W * q)) & ((1u << W) - 1u);
            const int ju = m.rj[uu];
            V acc[W];
#pragma unroll
            for (int t = 0; t < W; ++t) acc[t] = cmake<R>(0, 0);
            q_column<R, W>(Tq + ju * n2p, m.rj, tile + W * q, na, nlw, acc);   // mode D-2
            const V* xrow = tile + uu * nlw;
            {   // mode D-1 over the row's active span
                const int slo = __ffs(rb) - 1, shi = 31 - __clz(rb);
                for (int sp = slo; sp <= shi; ++sp) {
                    const V x = xrow[sp];
                    R tq[W];
                    ld_real_w<R, W>(Tlq + sp * nlw + W * q, tq);
#pragma unroll
                    for (int t = 0; t < W; ++t) {
                        cfma(acc[t], tq[t], x);
                    }
                }
            }
            {   // potential
                R vv[W];
                ld_real_w<R, W>(gs + W * q, vv);
                const R f = fj[uu];
#pragma unroll
                for (int t = 0; t < W; ++t) vv[t] += f;
                for (int tt = g3; tt < nt; ++tt) {
                    const R pj = pref[tt] * a.pot[((size_t)tt * D + D - 2) * kMaxN + ju];
                    R pl[W];
                    ld_real_w<R, W>(potl + (tt - g3) * nlw + W * q, pl);
#pragma unroll
                    for (int t = 0; t < W; ++t) vv[t] += pj * pl[t];
                }
                V x[W];
                ld_w<R, W>(xrow + W * q, x);
#pragma unroll
                for (int t = 0; t < W; ++t) {
                    cfma(acc[t], vv[t], x[t]);
                }
            }
            uint32_t p = m.rst[uu] + (uint32_t)__popc(rb & ((1u << (W * q)) - 1u));
#pragma unroll
            for (int t = 0; t < W; ++t) {
                if ((bq >> t) & 1u) {
                    if (pq_in_bounds(p, nact, 28, a.cnt)) a.out[p] = acc[t];
                    ++p;
                }
            }
        }
        __syncwarp();
    }
}

template <typename R, int W>
static size_t smem_inner_q(int n2, int nl, int nboth) {
    const int nlw = q_items_per_row(nl, W) * W;
    return (size_t)kQWarps * n2 * nlw * 2 * sizeof(R) +
           ((size_t)nl * nlw + (size_t)nboth * nlw + (size_t)n2 * (n2 | 1)) * sizeof(R);
}

static size_t smem_inner(const Lattice& L, int nterms, int wpb, size_t esz) {
    const int n2 = L.n[L.D - 2], nl = L.nlast;
    const size_t per_warp = (size_t)n2 * nl * 2 * esz + kMaxNTile * 8 + kMaxNTile * 4 + kMaxTerms * esz;
    const size_t shared = ((size_t)n2 * n2 + (size_t)nl * nl + (size_t)nterms * (n2 + nl)) * esz;
    return per_warp * wpb + shared;
}
static size_t smem_outer(const Lattice& L, int k, int wpb, size_t esz) {
    const int nk = L.n[k], nl = L.nlast;
    const size_t per_warp = (size_t)nk * nl * 2 * esz + kMaxNTile * 8 + kMaxNTile * 4;
    return per_warp * wpb + (size_t)nk * nk * esz;
}


template <typename R, int N2, int NL>
static pq_status launch_inner_reg(ApplyArgs<R> a, int G, cudaStream_t st) {
    const size_t esz = sizeof(R);
    const int wpb = kApplyThreads / 32;
    const size_t sm = (size_t)N2 * N2 * esz +
                      (size_t)wpb * ((size_t)N2 * NL * 2 * esz + N2 * 8 + N2 * 4 + kMaxTerms * esz + N2 * esz);
    static bool attr = false;
    if (!attr) {
        PQ_CUDA_TRY(cudaFuncSetAttribute(k_apply_inner_reg<R, N2, NL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    a.wpb = wpb;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_inner_reg<R, N2, NL>, kApplyThreads, sm);
    k_apply_inner_reg<R, N2, NL><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
    PQ_CHECK_LAUNCH();
    return PQ_OK;
}

template <typename R, int NK>
static pq_status launch_outer_reg(ApplyArgs<R> a, int G, cudaStream_t st) {
    const size_t esz = sizeof(R);
    const int wpb = kApplyThreads / 32;
    const size_t sm = (size_t)NK * NK * esz + (size_t)wpb * (NK * 8 + NK * 4);
    a.wpb = wpb;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_outer_reg<R, NK>, kApplyThreads, sm);
    k_apply_outer_reg<R, NK><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
    PQ_CHECK_LAUNCH();
    return PQ_OK;
}



// ------------------------------------------------------------------------
// Point-parallel pass for lattices with a mode longer than the tiled kernels
// take (n > 64, e.g. the FGH grids of the double well, Sec. 3.1): one thread
// per active point forms the whole pruned product for its point, every mode's
// fibre found by bitmap tests and rank queries on the fly, the SoP potential
// evaluated from the per-mode tables.  Meant for small lattices.
template <typename R>
__global__ void __launch_bounds__(256) k_apply_point(ApplyArgs<R> a) {
    using V = typename Cx<R>::T;
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.cnt[CNT_ERR] & 1) return;
    const Lattice& L = a.L;
    const int D = L.D, nt = a.nterms;
    const int64_t n = a.cnt[CNT_NA];
    const R scale = a.in_scale ? (R)(*a.in_scale) : (R)1;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = a.keys[p];
        int dg[kMaxD];
        for (int k = 0; k < D; ++k) dg[k] = (int)((key / L.stride[k]) % (uint32_t)L.n[k]);
        R vv = 0;
        for (int t = 0; t < nt; ++t) {
            R f = a.potc[t];
            for (int k = 0; k < D; ++k) f *= a.pot[((size_t)t * D + k) * kMaxN + dg[k]];
            vv += f;
        }
        const V xp = a.in[p];
        R ax = vv * xp.x, ay = vv * xp.y;
        for (int k = 0; k < D; ++k) {
            const uint32_t sk = L.stride[k];
            const uint32_t base = key - (uint32_t)dg[k] * sk;
            const R* trow = a.T + ((size_t)k * kMaxN + dg[k]) * kMaxN;
            for (int j = 0; j < L.n[k]; ++j) {
                const uint32_t q = base + (uint32_t)j * sk;
                if (!bit_test(a.bits, q)) continue;
                const uint32_t pos = rank_of(a.bits, a.off, q);
                if (!pq_in_bounds(pos, (uint64_t)n, 29, a.cnt)) continue;
                const V x = a.in[pos];
                ax += trow[j] * x.x;
                ay += trow[j] * x.y;
            }
        }
        a.out[p] = cmake<R>(scale * ax, scale * ay);
    }
}

template <typename R>
static pq_status launch_all(const State& s, const void* in, void* out, const double* in_scale,
                            const int* skip, int skip_k, cudaStream_t st) {
    const Lattice& L = s.lat;
    const size_t esz = sizeof(R);
    ApplyArgs<R> a{};
    a.L = L;
    a.bits = s.bits;
    a.off = s.off;
    a.in = (const typename Cx<R>::T*)in;
    a.out = (typename Cx<R>::T*)out;
    a.in_scale = in_scale;
    a.skip = skip;
    a.skip_k = skip_k;
    a.T = sizeof(R) == 8 ? (const R*)s.T64 : (const R*)s.T32;
    a.pot = sizeof(R) == 8 ? (const R*)s.pot64 : (const R*)s.pot32;
    a.potc = a.pot + (size_t)std::max(s.nterms, 1) * L.D * kMaxN;
    a.rowinfo = s.rowinfo;
    for (int g = 0; g < 4; ++g) a.ngroup[g] = s.ngroup[g];
    a.nterms = s.nterms;
    a.cnt = s.cnt;
    if (s.generic) return launch_generic<R>(s, a, in, out, in_scale, st);
    bool big = false;
    for (int k = 0; k < L.D; ++k) big = big || L.n[k] > kMaxNTile;
    if (big) {   // a mode longer than the tiled kernels take
        a.keys = s.keys;
        k_apply_point<R><<<grid_size() * 8, 256, 0, st>>>(a);
        PQ_CHECK_LAUNCH();
        return PQ_OK;
    }
    static bool attr_set[2][2] = {{false, false}, {false, false}};
    const int pi = sizeof(R) == 8 ? 1 : 0;
    if (!attr_set[pi][0]) {
        PQ_CUDA_TRY(cudaFuncSetAttribute(k_apply_inner<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        PQ_CUDA_TRY(cudaFuncSetAttribute(k_apply_outer<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        attr_set[pi][0] = true;
    }
    const int G = grid_size();
    static bool cmp_attr[2] = {false, false};
    if (!cmp_attr[pi]) {
        PQ_CUDA_TRY(cudaFuncSetAttribute(k_apply_inner_cmp<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        PQ_CUDA_TRY(cudaFuncSetAttribute(k_apply_outer_cmp<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        cmp_attr[pi] = true;
    }
    const bool compact = L.nlast <= 32;
    // Dense-tile passes (FP32): launched beside the item-blocked kernels, whose
    // conditions must then hold for every pass (they honour the gate); pairs
    // of outer modes from the top, (D-4, D-3), (D-6, D-5), ...
    bool use_dense = false;
    bool paired[kMaxD] = {false};
    if constexpr (std::is_same<R, float>::value) {
        const int n2 = L.n[L.D - 2], nl = L.nlast;
        const int nboth = s.nterms - (s.ngroup[0] + s.ngroup[1] + s.ngroup[2]);
        use_dense = s.rowinfo && dense_ok(L, s.nterms) && !s.vgrid32 && n2 <= 32 &&
                    smem_inner_q<R, kQWInner>(n2, nl, nboth) <= kSmemBudget;
        for (int k = 0; k + 2 < L.D && use_dense; ++k)
            use_dense = L.n[k] <= 32 && smem_outer_q<R, kQWOuter>(L.n[k], nl) <= kSmemBudget;
        if (use_dense)
            for (int k = L.D - 4; k >= 0; k -= 2)
                if (L.n[k] % 4 == 0 && smem_dense_pair(L, k) <= kSmemBudget) paired[k] = paired[k + 1] = true;
    }
    const int hint = use_dense ? s.dense_hint : 0;
    const bool run_sparse = hint != 1, run_dense = use_dense && hint != 0;
    const int gate = hint < 0 ? 1 : 0;   // both paths launched: the device picks
    // inner pass
    a.full_gate = -gate;
    if (run_sparse) {
        a.units = s.planes;
        a.units_cap = s.rows_cap;
        a.nunits = s.cnt + CNT_PLANES;
        int wpb = kApplyThreads / 32;
        const int n2 = L.n[L.D - 2], nl = L.nlast;
        const int nboth = s.nterms - (s.ngroup[0] + s.ngroup[1] + s.ngroup[2]);
        if (sizeof(R) == 4 && n2 <= 32 && nl <= 32 &&
            smem_inner_q<R, kQWInner>(n2, nl, nboth) <= kSmemBudget) {
            static bool q_attr[2] = {false, false};
            if (!q_attr[pi]) {
                PQ_CUDA_TRY(cudaFuncSetAttribute(k_inner_q<R, kQWInner>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmemBudget));
                q_attr[pi] = true;
            }
            const size_t sm = smem_inner_q<R, kQWInner>(n2, nl, nboth);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inner_q<R, kQWInner>, kApplyThreads, sm);
            k_inner_q<R, kQWInner><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
            PQ_CHECK_LAUNCH();
        } else if (n2 <= 32 && nl <= 32 && smem_inner_ep<R>(n2, nl) <= kSmemBudget) {
            static bool ep_attr[2] = {false, false};
            if (!ep_attr[pi]) {
                PQ_CUDA_TRY(cudaFuncSetAttribute(k_inner_ep<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmemBudget));
                ep_attr[pi] = true;
            }
            const size_t sm = smem_inner_ep<R>(n2, nl);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inner_ep<R>, kApplyThreads, sm);
            k_inner_ep<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
            PQ_CHECK_LAUNCH();
        } else if (n2 == nl && (nl == 16 || nl == 24 || nl == 32)) {
            pq_status rc = nl == 16 ? launch_inner_reg<R, 16, 16>(a, G, st)
                         : nl == 24 ? launch_inner_reg<R, 24, 24>(a, G, st)
                                    : launch_inner_reg<R, 32, 32>(a, G, st);
            if (rc) return rc;
        } else if (compact) {
            while (wpb > 1 && smem_inner_cmp<R>(n2, L.nlast, wpb) > kSmemBudget) --wpb;
            const size_t sm = smem_inner_cmp<R>(n2, L.nlast, wpb);
            a.wpb = wpb;
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_inner_cmp<R>, kApplyThreads, sm);
            k_apply_inner_cmp<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
            PQ_CHECK_LAUNCH();
        } else {
            while (wpb > 1 && smem_inner(L, s.nterms, wpb, esz) > kSmemBudget) --wpb;
            const size_t sm = smem_inner(L, s.nterms, wpb, esz);
            a.wpb = wpb;
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_inner<R>, kApplyThreads, sm);
            k_apply_inner<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
            PQ_CHECK_LAUNCH();
        }
    }
    if constexpr (std::is_same<R, float>::value) {
        if (run_dense) {
            static bool d_attr = false;
            if (!d_attr) {
                PQ_CUDA_TRY(cudaFuncSetAttribute(k_dense_inner, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmemBudget));
                PQ_CUDA_TRY(cudaFuncSetAttribute(k_dense_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmemBudget));
                d_attr = true;
            }
            ApplyArgs<float> ad = a;
            ad.full_gate = gate;
            const size_t smi = smem_dense_inner(L, s.nterms);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_inner, kDenseThreads, smi);
            k_dense_inner<<<G * (per_sm > 0 ? per_sm : 1), kDenseThreads, smi, st>>>(ad);
            PQ_CHECK_LAUNCH();
            for (int k = L.D - 4; k >= 0; k -= 2) {
                if (!paired[k]) continue;
                ad.mode = k;
                const size_t smp = smem_dense_pair(L, k);
                per_sm = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_pair, kDenseThreads, smp);
                k_dense_pair<<<G * (per_sm > 0 ? per_sm : 1), kDenseThreads, smp, st>>>(ad);
                PQ_CHECK_LAUNCH();
            }
        }
    }
    for (int k = L.D - 3; k >= 0; --k) {
        if (paired[k] && !run_sparse) continue;   // the dense pair pass covers it
        a.mode = k;
        a.full_gate = paired[k] ? -gate : 0;
        a.units = s.leaders + (size_t)k * s.rows_cap;
        a.units_cap = s.rows_cap;
        a.nunits = s.cnt + CNT_LEAD0 + k;
        int wpb = kApplyThreads / 32;
        const int nk = L.n[k];
        if (sizeof(R) == 4 && L.nlast <= 32 && nk <= 32 &&
            smem_outer_q<R, kQWOuter>(nk, L.nlast) <= kSmemBudget) {
            static bool q_attr[2] = {false, false};
            if (!q_attr[pi]) {
                PQ_CUDA_TRY(cudaFuncSetAttribute(k_outer_q<R, kQWOuter>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmemBudget));
                q_attr[pi] = true;
            }
            const size_t sm = smem_outer_q<R, kQWOuter>(nk, L.nlast);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_outer_q<R, kQWOuter>, kApplyThreads, sm);
            k_outer_q<R, kQWOuter><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
            PQ_CHECK_LAUNCH();
            continue;
        }
        if (L.nlast <= 32 && nk <= 32 && smem_outer_ep<R>(nk, L.nlast) <= kSmemBudget) {
            static bool ep_attr[2] = {false, false};
            if (!ep_attr[pi]) {
                // the batch metadata is static shared memory: leave room for it
                PQ_CUDA_TRY(cudaFuncSetAttribute(k_outer_ep<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmemBudget));
                ep_attr[pi] = true;
            }
            const size_t sm = smem_outer_ep<R>(nk, L.nlast);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_outer_ep<R>, kApplyThreads, sm);
            k_outer_ep<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
            PQ_CHECK_LAUNCH();
            continue;
        }
        if (L.nlast <= 32 && (nk == 16 || nk == 24 || nk == 32)) {
            pq_status rc = nk == 16 ? launch_outer_reg<R, 16>(a, G, st)
                         : nk == 24 ? launch_outer_reg<R, 24>(a, G, st)
                                    : launch_outer_reg<R, 32>(a, G, st);
            if (rc) return rc;
            continue;
        }
        if (compact) {
            while (wpb > 1 && smem_outer_cmp<R>(L.n[k], wpb) > kSmemBudget) --wpb;
            const size_t sm = smem_outer_cmp<R>(L.n[k], wpb);
            a.wpb = wpb;
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_outer_cmp<R>, kApplyThreads, sm);
            k_apply_outer_cmp<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
            PQ_CHECK_LAUNCH();
            continue;
        }
        while (wpb > 1 && smem_outer(L, k, wpb, esz) > kSmemBudget) --wpb;
        const size_t sm = smem_outer(L, k, wpb, esz);
        a.wpb = wpb;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_outer<R>, kApplyThreads, sm);
        k_apply_outer<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
        PQ_CHECK_LAUNCH();
    }
    return PQ_OK;
}

// out_I += V_grid(I) in_I for a tabulated (non-SoP) diagonal potential
// (Sec. 2.1: the DVR potential is diagonal): one thread per active point.
template <typename R>
__global__ void k_add_grid_potential(const uint32_t* __restrict__ keys, const int64_t* na,
                                     int64_t cap, const R* __restrict__ vgrid,
                                     const typename Cx<R>::T* __restrict__ in,
                                     typename Cx<R>::T* out, const double* in_scale,
                                     const int* skip, int skip_k) {
    using V = typename Cx<R>::T;
    if (skip && *skip <= skip_k) return;
    const int64_t n = min(*na, cap);
    const R scale = in_scale ? (R)(*in_scale) : (R)1;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const R v = vgrid[keys[p]] * scale;
        const V x = in[p];
        V o = out[p];
        o.x += v * x.x;
        o.y += v * x.y;
        out[p] = o;
    }
}

template <typename R>
static pq_status add_grid_potential(const State& s, const void* in, void* out,
                                    const double* in_scale, const int* skip, int skip_k,
                                    cudaStream_t st) {
    k_add_grid_potential<R><<<grid_size() * 8, 256, 0, st>>>(
        s.keys, s.cnt + CNT_NA, (int64_t)s.cap,
        sizeof(R) == 8 ? (const R*)s.vgrid64 : (const R*)s.vgrid32,
        (const typename Cx<R>::T*)in, (typename Cx<R>::T*)out, in_scale, skip, skip_k);
    PQ_CHECK_LAUNCH();
    return PQ_OK;
}

pq_status apply_H_launch(const State& s, const void* in, void* out, int prec,
                         const double* in_scale, const int* skip, int skip_k, cudaStream_t st) {
    if (s.pvb) {   // H_AA on the full grid (pvb.cu); called only from the C ABI
        if (in_scale || skip) {
            set_error("internal: scaled / skipped H.psi is not defined for pvB");
            return PQ_EINVAL;
        }
        return pvb_apply(const_cast<State&>(s), in, out, prec, st);
    }
    if (prec == PQ_FP64) {
        pq_status rc = launch_all<double>(s, in, out, in_scale, skip, skip_k, st);
        if (rc || !s.vgrid64) return rc;
        return add_grid_potential<double>(s, in, out, in_scale, skip, skip_k, st);
    }
    if (prec == PQ_FP32MIX) {
        pq_status rc = launch_all<float>(s, in, out, in_scale, skip, skip_k, st);
        if (rc || !s.vgrid32) return rc;
        return add_grid_potential<float>(s, in, out, in_scale, skip, skip_k, st);
    }
    set_error("unknown precision %d", prec);
    return PQ_EINVAL;
}

}  // namespace pq
