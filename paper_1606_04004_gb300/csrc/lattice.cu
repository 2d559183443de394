// Active-set maintenance on the device: the rank/select bitmap over the
// direct-product lattice, order-preserving compaction (reduce-then-scan with
// a fixed grid and device-resident sizes, no host round trip), the adaption
// of Sec. 2.5 (threshold + nearest-neighbour add, Sec. 3.1) and the tables the
// fibre transforms need (rows, planes, fibre leaders; Appendix: the per-mode
// fibre structure rebuilt whenever the basis changes).
#include <stdio.h>

#include <cmath>
#include <cstddef>

#include "device_util.cuh"

namespace pq {

constexpr int kScanBlocks = 1024;
constexpr int kScanThreads = 256;

int grid_size() {
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = sms > 0 ? sms : 132;
    }
    return g;
}

// ---------------------------------------------------------------- scans
// Op: __device__ int64_t size() const; uint32_t count(int64_t i) const;
//     void emit(int64_t i, uint32_t pos, uint32_t c) const.
template <class Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_count(Op op, uint32_t* block_sums) {
    __shared__ uint32_t sh[32];
    const int64_t n = op.size();
    const int64_t seg = (n + gridDim.x - 1) / gridDim.x;
    const int64_t start = (int64_t)blockIdx.x * seg;
    const int64_t end = min(n, start + seg);
    uint32_t local = 0;
    for (int64_t i = start + threadIdx.x; i < end; i += blockDim.x) local += op.count(i);
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) block_sums[blockIdx.x] = v;
    }
}

// One block: exclusive scan of the G block sums in place; total -> *total.
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t* block_sums, int G,
                                                      int64_t* total, int64_t cap,
                                                      int64_t* err, int errbit) {
    __shared__ uint32_t sh[32];
    uint32_t carry = 0;
    for (int base = 0; base < G; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < G ? block_sums[i] : 0;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, sh, &tot);
        if (i < G) block_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *total = carry;
        if (cap >= 0 && (int64_t)carry > cap && err) *err |= errbit;
    }
}

template <class Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_emit(Op op, const uint32_t* block_sums) {
    __shared__ uint32_t sh[32];
    const int64_t n = op.size();
    const int64_t seg = (n + gridDim.x - 1) / gridDim.x;
    const int64_t start = (int64_t)blockIdx.x * seg;
    const int64_t end = min(n, start + seg);
    uint32_t base = block_sums[blockIdx.x];
    for (int64_t t0 = start; t0 < end; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        const uint32_t c = i < end ? op.count(i) : 0;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(c, sh, &tot);
        if (i < end) op.emit(i, base + ex, c);
        base += tot;
    }
}

template <class Op>
static pq_status run_scan(const Op& op, uint32_t* scan_tmp, int64_t* total, int64_t cap,
                          int64_t* err, int errbit, cudaStream_t st) {
    k_scan_count<Op><<<kScanBlocks, kScanThreads, 0, st>>>(op, scan_tmp);
    PQ_CHECK_LAUNCH();
    k_scan_blocks<<<1, 1024, 0, st>>>(scan_tmp, kScanBlocks, total, cap, err, errbit);
    PQ_CHECK_LAUNCH();
    k_scan_emit<Op><<<kScanBlocks, kScanThreads, 0, st>>>(op, scan_tmp);
    PQ_CHECK_LAUNCH();
    return PQ_OK;
}

// Bitmap words -> rank offsets and the sorted key list.
struct OpWords {
    const uint64_t* bits;
    uint32_t* off;
    uint32_t* keys;
    uint32_t nwords;
    int64_t cap;
    __device__ int64_t size() const { return nwords; }
    __device__ uint32_t count(int64_t w) const { return __popcll(bits[w]); }
    __device__ void emit(int64_t w, uint32_t pos, uint32_t c) const {
        off[w] = pos;
        if (w == nwords - 1) off[nwords] = pos + c;
        uint64_t b = bits[w];
        uint32_t p = pos;
        while (b) {
            const int t = __ffsll((long long)b) - 1;
            if ((int64_t)p < cap) keys[p] = (uint32_t)(w * 64 + t);
            ++p;
            b &= b - 1;
        }
    }
};

// Keys -> active rows (first point of each row).
struct OpRows {
    const uint32_t* keys;
    const int64_t* na;
    uint32_t* rows;
    int nlast;
    int64_t cap;
    uint64_t rows_cap;
    int64_t* cnt;
    __device__ int64_t size() const { return min(*na, cap); }
    __device__ uint32_t count(int64_t p) const {
        return p == 0 || keys[p] / nlast != keys[p - 1] / nlast;
    }
    __device__ void emit(int64_t p, uint32_t pos, uint32_t c) const {
        if (c && pq_in_bounds(pos, rows_cap, 8, cnt)) rows[pos] = keys[p] / nlast;
    }
};

// Rows -> active planes (rows sharing all digits but the last two).
struct OpPlanes {
    const uint32_t* rows;
    const int64_t* nr;
    uint32_t* planes;
    int n2;
    uint64_t rows_cap;
    int64_t* cnt;
    __device__ int64_t size() const { return *nr; }
    __device__ uint32_t count(int64_t u) const {
        return u == 0 || rows[u] / n2 != rows[u - 1] / n2;
    }
    __device__ void emit(int64_t u, uint32_t pos, uint32_t c) const {
        if (c && pq_in_bounds(pos, rows_cap, 9, cnt)) planes[pos] = rows[u] / n2;
    }
};

// Rows -> fibre leaders of outer mode k: the active row with the smallest
// digit i_k among the rows that differ from it only in digit k.
struct OpLeaders {
    const uint32_t* rows;
    const int64_t* nr;
    const uint64_t* bits;
    uint32_t* out;
    uint32_t rstride;
    int nk, nlast;
    uint64_t rows_cap;
    int64_t* cnt;
    __device__ int64_t size() const { return *nr; }
    __device__ uint32_t count(int64_t u) const {
        const uint32_t r = rows[u];
        const int ik = (int)((r / rstride) % (uint32_t)nk);
        for (int j = 1; j <= ik; ++j)
            if (row_bits(bits, r - (uint32_t)j * rstride, nlast)) return 0;
        return 1;
    }
    __device__ void emit(int64_t u, uint32_t pos, uint32_t c) const {
        if (c && pq_in_bounds(pos, rows_cap, 10, cnt)) out[pos] = rows[u];
    }
};

// Carry coefficients from the old active set (old bitmap + rank) to the new.
template <typename V>
__global__ void k_remap(const uint32_t* __restrict__ keys, const int64_t* na, int64_t cap,
                        const uint64_t* __restrict__ obits, const uint32_t* __restrict__ ooff,
                        const V* __restrict__ opsi, V* __restrict__ npsi, int64_t* cnt) {
    if (cnt[CNT_ERR] & 1) return;   // capacity overflow: positions are not valid
    const int64_t n = min(*na, cap);
#ifdef PQ_BOUNDS_CHECK
    const uint64_t nold = (uint64_t)cnt[CNT_NA_OLD];
#else
    const uint64_t nold = 0;
#endif
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[p];
        V v;
        v.x = 0;
        v.y = 0;
        if (bit_test(obits, k)) {
            const uint32_t r = rank_of(obits, ooff, k);
            if (pq_in_bounds(r, nold, 7, cnt)) v = opsi[r];
        }
        npsi[p] = v;
    }
}

// rowinfo[r] = (rank of the row's first bit, the row's active pattern) for
// every active row r (empty rows were cleared to (0, 0)).
__global__ void k_fill_rowinfo(const uint32_t* __restrict__ rows, const int64_t* nr,
                               const uint64_t* __restrict__ bits, const uint32_t* __restrict__ off,
                               int nlast, uint2* rowinfo) {
    const int64_t n = *nr;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = rows[u];
        const uint64_t b = row_bits(bits, r, nlast);
        rowinfo[r] = make_uint2(rank_of(bits, off, (uint64_t)r * nlast), (uint32_t)b);
    }
}

pq_status rebuild_tables(State& s, cudaStream_t st) {
    const Lattice& L = s.lat;
    pq_status rc;
    OpRows orow{s.keys, s.cnt + CNT_NA, s.rows, L.nlast, (int64_t)s.cap, s.rows_cap, s.cnt};
    if ((rc = run_scan(orow, s.scan_tmp, s.cnt + CNT_ROWS, -1, nullptr, 0, st))) return rc;
    if (s.rowinfo) {
        PQ_CUDA_TRY(cudaMemsetAsync(s.rowinfo, 0, (size_t)L.nrows * sizeof(uint2), st));
        k_fill_rowinfo<<<grid_size() * 8, 256, 0, st>>>(s.rows, s.cnt + CNT_ROWS, s.bits, s.off,
                                                       L.nlast, s.rowinfo);
        PQ_CHECK_LAUNCH();
    }
    OpPlanes opl{s.rows, s.cnt + CNT_ROWS, s.planes, L.n[L.D - 2], s.rows_cap, s.cnt};
    if ((rc = run_scan(opl, s.scan_tmp, s.cnt + CNT_PLANES, -1, nullptr, 0, st))) return rc;
    if (L.nlast > kMaxNTile) {   // fibre leaders serve the tiled kernels only
        PQ_CUDA_TRY(cudaMemsetAsync(s.cnt + CNT_LEAD0, 0, sizeof(int64_t) * (kMaxD - 1), st));
        return PQ_OK;
    }
    // fibre leaders of every mode but the last; a DVR Hamiltonian's passes take
    // mode D-2 in the inner pass (planes), so its leaders serve only the
    // generic (phase-space) passes
    const int kend = s.generic ? L.D - 1 : L.D - 2;
    PQ_CUDA_TRY(cudaMemsetAsync(s.cnt + CNT_LEAD0 + std::max(kend, 0), 0,
                                sizeof(int64_t) * (size_t)(L.D - 1 - std::max(kend, 0)), st));
    for (int k = 0; k < kend; ++k) {
        OpLeaders ol{s.rows, s.cnt + CNT_ROWS, s.bits, s.leaders + (size_t)k * s.rows_cap,
                     L.rstride[k], L.n[k], L.nlast, s.rows_cap, s.cnt};
        if ((rc = run_scan(ol, s.scan_tmp, s.cnt + CNT_LEAD0 + k, -1, nullptr, 0, st))) return rc;
    }
    return PQ_OK;
}

// Rebuild keys / rank / tables after the bitmap `bits_alt` was filled.  With
// `remap`, coefficients are carried over from the current (bits, off, psi)
// into psi_alt; afterwards the buffers are swapped so that the new set is
// current.
pq_status rebuild_from_bits(State& s, bool remap, cudaStream_t st) {
    const Lattice& L = s.lat;
    PQ_CUDA_TRY(cudaMemcpyAsync(s.cnt + CNT_NA_OLD, s.cnt + CNT_NA, sizeof(int64_t),
                                cudaMemcpyDeviceToDevice, st));
    OpWords ow{s.bits_alt, s.off_alt, s.keys, L.nwords, (int64_t)s.cap};
    pq_status rc = run_scan(ow, s.scan_tmp, s.cnt + CNT_NA, (int64_t)s.cap, s.cnt + CNT_ERR, 1, st);
    if (rc) return rc;
    if (remap) {
        const int G = grid_size() * 8;
        if (s.prec == PQ_FP64)
            k_remap<double2><<<G, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap, s.bits,
                                                s.off, (const double2*)s.psi, (double2*)s.psi_alt, s.cnt);
        else
            k_remap<float2><<<G, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap, s.bits,
                                               s.off, (const float2*)s.psi, (float2*)s.psi_alt, s.cnt);
        PQ_CHECK_LAUNCH();
        void* t = s.psi;
        s.psi = s.psi_alt;
        s.psi_alt = t;
    }
    uint64_t* tb = s.bits;
    s.bits = s.bits_alt;
    s.bits_alt = tb;
    uint32_t* to = s.off;
    s.off = s.off_alt;
    s.off_alt = to;
    return rebuild_tables(s, st);
}

// ------------------------------------------------------------- adaption
// Neighbour rules of Sec. 3.1 on the lattice axes ("phase-space ball radius"):
// PQ_RADIUS_1 moves +-1 along one axis (2k neighbours on k axes),
// PQ_RADIUS_SQRT2 also along two axes at once (2k^2), PQ_RADIUS_2 along any
// number of axes (3^k - 1).  Neighbours outside the lattice are dropped.
__device__ __forceinline__ void mark_with_neighbours(uint64_t* bits, uint32_t key,
                                                     const Lattice& L, int rule) {
    bit_mark(bits, key);
    int dg[2 * kMaxD];
    for (int a = 0; a < L.naxes; ++a) dg[a] = (int)((key / L.axis_stride[a]) % (uint32_t)L.axis_n[a]);
    for (int a = 0; a < L.naxes; ++a) {
        const uint32_t sa = L.axis_stride[a];
        if (dg[a] > 0) bit_mark(bits, key - sa);
        if (dg[a] + 1 < L.axis_n[a]) bit_mark(bits, key + sa);
    }
    if (rule == PQ_RADIUS_SQRT2) {
        for (int a = 0; a < L.naxes; ++a)
            for (int b = a + 1; b < L.naxes; ++b)
                for (int sa = -1; sa <= 1; sa += 2)
                    for (int sb = -1; sb <= 1; sb += 2) {
                        const int da = dg[a] + sa, db = dg[b] + sb;
                        if (da < 0 || da >= L.axis_n[a] || db < 0 || db >= L.axis_n[b]) continue;
                        bit_mark(bits, key + (uint32_t)(sa * (int64_t)L.axis_stride[a] +
                                                       sb * (int64_t)L.axis_stride[b]));
                    }
    } else if (rule == PQ_RADIUS_2) {
        // offsets in {-1, 0, 1}^k, counted in base 3 (digit 0 -> -1, 1 -> 0, 2 -> +1)
        int c[2 * kMaxD];
        for (int a = 0; a < L.naxes; ++a) c[a] = 0;
        while (true) {
            int moved = 0;
            bool ok = true;
            int64_t delta = 0;
            for (int a = 0; a < L.naxes; ++a) {
                const int o = c[a] - 1;
                if (o) {
                    ++moved;
                    const int d = dg[a] + o;
                    ok = ok && d >= 0 && d < L.axis_n[a];
                    delta += o * (int64_t)L.axis_stride[a];
                }
            }
            if (ok && moved >= 2) bit_mark(bits, (uint32_t)((int64_t)key + delta));
            int a = 0;   // next offset
            while (a < L.naxes && c[a] == 2) c[a++] = 0;
            if (a == L.naxes) break;
            ++c[a];
        }
    }
}

template <typename R>
__global__ void k_prune_mark(const uint32_t* __restrict__ keys, const int64_t* na, int64_t cap,
                             const typename Cx<R>::T* __restrict__ psi, double theta2,
                             float lo, float hi, Lattice L, int rule, uint64_t* bits,
                             const int64_t* cnt) {
    if (cnt[CNT_ERR] & 1) return;
    const int64_t n = min(*na, cap);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const auto v = psi[p];
        bool sig;
        if (sizeof(R) == 8)
            sig = significant64((double)v.x, (double)v.y, theta2);
        else
            sig = significant32((float)v.x, (float)v.y, theta2, lo, hi);
        if (sig) mark_with_neighbours(bits, keys[p], L, rule);
    }
}

// Relative exclusion (Sec. 2.5): count the members of A that the new bitmap
// drops, then, if there are at most rel_excl * |A| of them, put them back.
__global__ void k_excl_count(const uint32_t* __restrict__ keys, const int64_t* na, int64_t cap,
                             const uint64_t* __restrict__ bits, int64_t* cnt) {
    if (cnt[CNT_ERR] & 1) return;
    const int64_t n = min(*na, cap);
    int64_t c = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        c += bit_test(bits, keys[p]) ? 0 : 1;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c)
        atomicAdd(reinterpret_cast<unsigned long long*>(cnt + CNT_EXCL), (unsigned long long)c);
}

__global__ void k_excl_keep(const uint32_t* __restrict__ keys, const int64_t* na, int64_t cap,
                            double rel_excl, uint64_t* bits, const int64_t* cnt) {
    if (cnt[CNT_ERR] & 1) return;
    const int64_t n = min(*na, cap);
    if ((double)cnt[CNT_EXCL] > rel_excl * (double)n) return;   // exclusion goes ahead
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        bit_set(bits, keys[p]);
}

static void guard_band(double theta2, float* lo, float* hi) {
    // FP32 estimate of |a|^2 has relative error < 3 * 2^-24; a 1e-5 band is
    // far wider.  Below the FP32 normal range, always fall back to FP64.
    if (theta2 < 1e-30) {
        *lo = -1.0f;
        *hi = 3.0e38f;
    } else {
        *lo = (float)(theta2 * (1.0 - 1e-5));
        *hi = (float)(theta2 * (1.0 + 1e-5));
    }
}

pq_status check_neighbour_rule(const Lattice& L, int radius) {
    if (radius != PQ_RADIUS_1 && radius != PQ_RADIUS_SQRT2 && radius != PQ_RADIUS_2) {
        set_error("unknown neighbour rule %d (1: radius 1, 2: radius sqrt 2, 3: radius 2)", radius);
        return PQ_EINVAL;
    }
    if (radius == PQ_RADIUS_2 && L.naxes > kMaxBoxAxes) {
        set_error("neighbour radius 2 adds 3^k - 1 points: at most %d lattice axes (%d given)",
                  kMaxBoxAxes, L.naxes);
        return PQ_ENOTSUP;
    }
    return PQ_OK;
}

pq_status prune_launch(State& s, double theta, int radius, double rel_excl, cudaStream_t st) {
    const Lattice& L = s.lat;
    pq_status rc = check_neighbour_rule(L, radius);
    if (rc) return rc;
    if (!(rel_excl >= 0) || !std::isfinite(rel_excl)) {
        set_error("relative exclusion threshold must be finite and >= 0");
        return PQ_EINVAL;
    }
    PQ_CUDA_TRY(cudaMemsetAsync(s.bits_alt, 0, (size_t)L.nwords * 8, st));
    const double theta2 = theta * theta;
    float lo, hi;
    guard_band(theta2, &lo, &hi);
    const int G = grid_size() * 8;
    if (s.prec == PQ_FP64)
        k_prune_mark<double><<<G, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap,
                                                (const double2*)s.psi, theta2, lo, hi, L, radius,
                                                s.bits_alt, s.cnt);
    else
        k_prune_mark<float><<<G, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap,
                                               (const float2*)s.psi, theta2, lo, hi, L, radius,
                                               s.bits_alt, s.cnt);
    PQ_CHECK_LAUNCH();
    if (rel_excl > 0.0) {
        PQ_CUDA_TRY(cudaMemsetAsync(s.cnt + CNT_EXCL, 0, sizeof(int64_t), st));
        k_excl_count<<<G, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap, s.bits_alt, s.cnt);
        PQ_CHECK_LAUNCH();
        k_excl_keep<<<G, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap, rel_excl,
                                       s.bits_alt, s.cnt);
        PQ_CHECK_LAUNCH();
    }
    return rebuild_from_bits(s, true, st);
}

// ------------------------------------------------ initial packet, loading
// Initial adaption over the full lattice: a0_I = prod_k f_k(i_k) (complex
// FP64, multiplied in mode order), S = {|a0_I| >= theta}, A = S + neighbours.
__global__ void k_init_mark(Lattice L, const double2* __restrict__ fac, double theta2,
                            int rule, uint64_t* bits) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)L.nfull;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = (uint32_t)i;
        double re = 1.0, im = 0.0;
        for (int k = 0; k < L.D; ++k) {
            const int d = (int)((key / L.stride[k]) % (uint32_t)L.n[k]);
            const double2 f = fac[k * kMaxN + d];
            const double nr = __dsub_rn(__dmul_rn(re, f.x), __dmul_rn(im, f.y));
            const double ni = __dadd_rn(__dmul_rn(re, f.y), __dmul_rn(im, f.x));
            re = nr;
            im = ni;
        }
        if (significant64(re, im, theta2)) mark_with_neighbours(bits, key, L, rule);
    }
}

template <typename V>
__global__ void k_packet_on_set(const uint32_t* __restrict__ keys, const int64_t* na,
                                int64_t cap, Lattice L, const double2* __restrict__ fac,
                                V* __restrict__ psi) {
    const int64_t n = min(*na, cap);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = keys[p];
        double re = 1.0, im = 0.0;
        for (int k = 0; k < L.D; ++k) {
            const int d = (int)((key / L.stride[k]) % (uint32_t)L.n[k]);
            const double2 f = fac[k * kMaxN + d];
            const double nr = __dsub_rn(__dmul_rn(re, f.x), __dmul_rn(im, f.y));
            const double ni = __dadd_rn(__dmul_rn(re, f.y), __dmul_rn(im, f.x));
            re = nr;
            im = ni;
        }
        V v;
        v.x = re;
        v.y = im;
        psi[p] = v;
    }
}

pq_status init_bits_from_packet(State& s, double theta, cudaStream_t st) {
    const Lattice& L = s.lat;
    PQ_CUDA_TRY(cudaMemsetAsync(s.bits_alt, 0, (size_t)L.nwords * 8, st));
    pq_status rc = check_neighbour_rule(L, s.radius);
    if (rc) return rc;
    k_init_mark<<<grid_size() * 16, 256, 0, st>>>(L, (const double2*)s.fac64, theta * theta,
                                                  s.radius, s.bits_alt);
    PQ_CHECK_LAUNCH();
    return rebuild_from_bits(s, false, st);
}

pq_status reset_norm_keeping(State& s, cudaStream_t st) {
    if (s.ks)
        PQ_CUDA_TRY(cudaMemsetAsync(reinterpret_cast<char*>(s.ks) + offsetof(KrylovScalars, renorm), 0,
                                    3 * sizeof(double), st));
    return PQ_OK;
}

pq_status set_psi_from_packet(State& s, cudaStream_t st) {
    const int G = grid_size() * 8;
    pq_status rc = reset_norm_keeping(s, st);   // a new state: no pending correction
    if (rc) return rc;
    if (s.prec == PQ_FP64)
        k_packet_on_set<double2><<<G, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap,
                                                    s.lat, (const double2*)s.fac64,
                                                    (double2*)s.psi);
    else
        k_packet_on_set<float2><<<G, 256, 0, st>>>(s.keys, s.cnt + CNT_NA, (int64_t)s.cap,
                                                   s.lat, (const double2*)s.fac64,
                                                   (float2*)s.psi);
    PQ_CHECK_LAUNCH();
    return PQ_OK;
}

__global__ void k_set_bits(const uint32_t* __restrict__ keys, int64_t n, uint64_t* bits) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        bit_set(bits, keys[p]);
}

// Replace the active set by n sorted distinct keys already on the device
// (d_keys may alias nothing of the state).
pq_status load_set(State& s, const uint32_t* d_keys, int64_t n, cudaStream_t st, bool remap) {
    const Lattice& L = s.lat;
    s.dense_hint = 2 * n >= (int64_t)L.nfull ? 1 : 0;
    if (!remap) {   // new coefficients: no pending FP32-mix norm correction
        pq_status rc = reset_norm_keeping(s, st);
        if (rc) return rc;
    }
    if (!remap) PQ_CUDA_TRY(cudaMemsetAsync(s.cnt + CNT_ERR, 0, sizeof(int64_t), st));
    PQ_CUDA_TRY(cudaMemsetAsync(s.bits_alt, 0, (size_t)L.nwords * 8, st));
    if (n > 0) {
        k_set_bits<<<grid_size() * 8, 256, 0, st>>>(d_keys, n, s.bits_alt);
        PQ_CHECK_LAUNCH();
    }
    return rebuild_from_bits(s, remap, st);
}

// -------------------------------------------------------------- setup
pq_status lattice_setup(State& s) {
    Lattice& L = s.lat;
    uint64_t full = 1;
    for (int k = L.D - 1; k >= 0; --k) {
        L.stride[k] = (uint32_t)full;
        full *= (uint64_t)L.n[k];
    }
    if (full >= (1ull << 32)) {
        set_error("lattice of %llu points needs 64-bit indices (limit 2^32)",
                  (unsigned long long)full);
        return PQ_EINVAL;
    }
    L.nfull = (uint32_t)full;
    L.nlast = L.n[L.D - 1];
    L.nrows = L.nfull / (uint32_t)L.nlast;
    L.nplanes = L.nrows / (uint32_t)L.n[L.D - 2];
    for (int k = 0; k < L.D - 1; ++k) L.rstride[k] = L.stride[k] / (uint32_t)L.nlast;
    for (int k = 0; k < L.D - 2; ++k)
        L.pstride[k] = L.stride[k] / ((uint32_t)L.nlast * (uint32_t)L.n[L.D - 2]);
    L.nwords = (uint32_t)((full + 63) / 64);
    return PQ_OK;
}

}  // namespace pq
