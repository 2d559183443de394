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
#include "device_util.cuh"

namespace pq {

constexpr int kApplyThreads = 256;

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
    const R* pot;               // [nterms][D][kMaxN]
    int nterms;
    int mode;                   // outer mode k (outer pass only)
    int wpb;                    // warps per block
    int64_t* cnt;               // state counters (bounds-check build)
    uint64_t units_cap;         // entries of the units array (bounds-check build)
};

__device__ __forceinline__ uint64_t low_mask(int s) {
    return s >= 64 ? ~0ull : ((1ull << s) - 1ull);
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
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + (size_t)kMaxN * a.wpb);
    R* pref_all = reinterpret_cast<R*>(rstart_all + (size_t)kMaxN * a.wpb);
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
    uint64_t* rbits = rbits_all + (size_t)kMaxN * w;
    uint32_t* rstart = rstart_all + (size_t)kMaxN * w;
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
            R p = (R)1;
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
    uint32_t* rstart_all = reinterpret_cast<uint32_t*>(rbits_all + (size_t)kMaxN * a.wpb);
    R* Tk = reinterpret_cast<R*>(rstart_all + (size_t)kMaxN * a.wpb);   // [nk][nk]
    for (int i = threadIdx.x; i < nk * nk; i += blockDim.x)
        Tk[i] = a.T[(size_t)k * kMaxN * kMaxN + (i / nk) * kMaxN + (i % nk)];
    __syncthreads();

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= a.wpb) return;
    V* tile = tiles + tile_elems * w;
    uint64_t* rbits = rbits_all + (size_t)kMaxN * w;
    uint32_t* rstart = rstart_all + (size_t)kMaxN * w;
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

static size_t smem_inner(const Lattice& L, int nterms, int wpb, size_t esz) {
    const int n2 = L.n[L.D - 2], nl = L.nlast;
    const size_t per_warp = (size_t)n2 * nl * 2 * esz + kMaxN * 8 + kMaxN * 4 + kMaxTerms * esz;
    const size_t shared = ((size_t)n2 * n2 + (size_t)nl * nl + (size_t)nterms * (n2 + nl)) * esz;
    return per_warp * wpb + shared;
}
static size_t smem_outer(const Lattice& L, int k, int wpb, size_t esz) {
    const int nk = L.n[k], nl = L.nlast;
    const size_t per_warp = (size_t)nk * nl * 2 * esz + kMaxN * 8 + kMaxN * 4;
    return per_warp * wpb + (size_t)nk * nk * esz;
}

constexpr size_t kSmemBudget = 200 * 1024;

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
    a.nterms = s.nterms;
    a.cnt = s.cnt;
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
    // inner pass
    {
        int wpb = kApplyThreads / 32;
        while (wpb > 1 && smem_inner(L, s.nterms, wpb, esz) > kSmemBudget) --wpb;
        const size_t sm = smem_inner(L, s.nterms, wpb, esz);
        a.wpb = wpb;
        a.units = s.planes;
        a.units_cap = s.rows_cap;
        a.nunits = s.cnt + CNT_PLANES;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_inner<R>, kApplyThreads, sm);
        k_apply_inner<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
        PQ_CHECK_LAUNCH();
    }
    for (int k = L.D - 3; k >= 0; --k) {
        int wpb = kApplyThreads / 32;
        while (wpb > 1 && smem_outer(L, k, wpb, esz) > kSmemBudget) --wpb;
        const size_t sm = smem_outer(L, k, wpb, esz);
        a.wpb = wpb;
        a.mode = k;
        a.units = s.leaders + (size_t)k * s.rows_cap;
        a.units_cap = s.rows_cap;
        a.nunits = s.cnt + CNT_LEAD0 + k;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_outer<R>, kApplyThreads, sm);
        k_apply_outer<R><<<G * (per_sm > 0 ? per_sm : 1), kApplyThreads, sm, st>>>(a);
        PQ_CHECK_LAUNCH();
    }
    return PQ_OK;
}

pq_status apply_H_launch(const State& s, const void* in, void* out, int prec,
                         const double* in_scale, const int* skip, int skip_k, cudaStream_t st) {
    if (prec == PQ_FP64) return launch_all<double>(s, in, out, in_scale, skip, skip_k, st);
    if (prec == PQ_FP32MIX) return launch_all<float>(s, in, out, in_scale, skip, skip_k, st);
    set_error("unknown precision %d", prec);
    return PQ_EINVAL;
}

}  // namespace pq
