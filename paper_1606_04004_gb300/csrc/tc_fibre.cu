// Dense 1D operators of the phase-space bases on the tensor cores (FP32-mix):
// a 64 x 64 (or smaller, zero-padded) matrix applied along one mode of
//   * the full grid (pvB, Sec. 2.2: the transforms by B, B^dagger, S and the
//     DVR kinetic matrix of y = P_A (x B^dagger) H^chi (x B) P_A^T a), or
//   * the pruned set (projected Weylets, Sec. 2.4 with the pruned sequential
//     transform of Sec. 2.2.2: out (+)= c P_A (h along mode k) in, the fibres
//     zero-padded to full length).
// Full fibres of 64 points form a real GEMM: 64 columns of complex data are
// 128 real rows (re, im) of the A operand, the fibre index is K, and the
// matrix is the B operand (N = 64 output points; N = 128 for a complex matrix,
// its real part in rows 0..63 and its imaginary part in rows 64..127, the
// complex product assembled in the epilogue).
//
// Precision: split TF32 (Ootomo and Yokota): a = a_hi + a_lo with a_hi the
// TF32 rounding of a and a_lo the TF32 rounding of a - a_hi, likewise for the
// matrix; D = A_hi B_hi accumulates in one TMEM tile and A_hi B_lo + A_lo B_hi
// in a second, summed in FP32 in the epilogue, so the products carry about
// FP32 accuracy (the dropped A_lo B_lo term is below 2^-21 relative).
//
// Per CTA (128 threads = the four TMEM lane quarters, persistent over tiles):
// threads stage a tile into shared memory in the K-major no-swizzle layout of
// 8-row x 16-byte core matrices; one thread issues tcgen05.mma (kind::tf32,
// M = 128, K = 8 per instruction) and commits to an mbarrier; every thread
// waits (bounded), reads its TMEM lane with tcgen05.ld and writes its outputs.
#include <algorithm>

#include "device_util.cuh"

namespace pq {

constexpr int kTcThreads = 128;
constexpr int kTcK = 64;                       // padded fibre length (K)
constexpr uint32_t kTcLBO = 128;               // K-adjacent core matrices
constexpr uint32_t kTcSBO = 16 * 128 + 16;     // 8-row groups (16 B skew against bank conflicts)
constexpr long long kTcWaitCycles = 4000000000ll;   // about 2 s at 2 GHz

enum : int { TC_DENSE = 0, TC_FIBRE = 1, TC_ROWS = 2 };

struct TcArgs {
    const float2* in;
    float2* out;
    const float* M;          // matrix, row stride kMaxN (complex interleaved when mcomplex)
    int mcomplex;
    int nk;                  // matrix size, <= 64
    float coef;
    int accumulate;
    const double* in_scale;
    const int* skip;
    int skip_k;
    // full grid
    uint32_t inner;          // stride of the mode
    uint32_t ncols;          // number of fibres (lattice size / nk)
    // pruned set
    Lattice L;
    const uint64_t* bits;
    const uint32_t* off;
    const uint32_t* units;   // fibre leaders (TC_FIBRE) or active rows (TC_ROWS)
    const int64_t* nunits;
    int mode;
    int64_t* cnt;            // state counters (error bit 4: a tensor-core wait gave up)
    const double* gate;      // nullable: nothing to do while *gate != 0
};

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row r, k) in a K-major, no-swizzle operand tile
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
    return (uint32_t)(r >> 3) * kTcSBO + (uint32_t)(k >> 2) * kTcLBO + (uint32_t)(r & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kTcLBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((kTcSBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tc_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       int accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            tc_smem(mbar))
        : "memory");
}

__device__ __forceinline__ bool tc_try_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(tc_smem(mbar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// 16 consecutive TMEM columns of this thread's lane, waited for in the same
// statement so that the values are complete when they are used
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared memory: A_hi, A_lo (128 rows), B_hi, B_lo (64 NMAT rows), per-tile
// row patterns and starts, the mbarrier and the TMEM address.
template <int NMAT>
struct TcSmem {
    static constexpr uint32_t kA = 16 * kTcSBO;          // 128 rows
    static constexpr uint32_t kB = 8 * NMAT * kTcSBO;    // 64 NMAT rows
    static constexpr uint32_t A_hi = 0, A_lo = kA, B_hi = 2 * kA, B_lo = 2 * kA + kB;
    static constexpr uint32_t rbits = 2 * kA + 2 * kB;   // uint64 [64]
    static constexpr uint32_t rst = rbits + 64 * 8;      // uint32 [64]
    static constexpr uint32_t mbar = rst + 64 * 4;       // uint64
    static constexpr uint32_t tslot = mbar + 8;          // uint32
    static constexpr uint32_t total = tslot + 8;
};

template <int NMAT, int GM>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_mode(const TcArgs a) {
    if (a.skip && *a.skip <= a.skip_k) return;
    if (a.gate && *a.gate != 0.0) return;
    if (a.cnt && (a.cnt[CNT_ERR] & 1)) return;
    using S = TcSmem<NMAT>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* rb = reinterpret_cast<uint64_t*>(smem + S::rbits);
    uint32_t* rs = reinterpret_cast<uint32_t*>(smem + S::rst);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::mbar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::tslot);
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr int N = 64 * NMAT;
    constexpr uint32_t kCols = 2 * N;   // TMEM columns: hi*hi, then the two cross terms
    const int nk = a.nk;
    const float scale = a.in_scale ? (float)(*a.in_scale) : 1.0f;
    int64_t ntiles;
    if (GM == TC_DENSE) ntiles = ((int64_t)a.ncols + 63) / 64;
    else if (GM == TC_FIBRE) ntiles = *a.nunits;
    else ntiles = (*a.nunits + 63) / 64;
    if ((int64_t)blockIdx.x >= ntiles) return;

    // ---- TMEM (one warp allocates), mbarrier, the matrix as B_hi / B_lo
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         tc_smem(tslot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int e = tid; e < N * kTcK; e += kTcThreads) {
        const int n = e / kTcK, k = e - n * kTcK;
        const int l = n & 63, part = n >> 6;   // part 1: imaginary part of a complex matrix
        float v = 0.f;
        if (l < nk && k < nk) {
            const size_t at = (size_t)l * kMaxN + k;
            v = a.mcomplex ? a.M[2 * at + part] : a.M[at];
        }
        const float hi = tc_tf32(v), lo = tc_tf32(v - hi);
        *reinterpret_cast<float*>(smem + S::B_hi + tc_off(n, k)) = hi;
        *reinterpret_cast<float*>(smem + S::B_lo + tc_off(n, k)) = lo;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);   // this warp's lane quarter
    const uint32_t idesc = tc_idesc(128, N);
    uint32_t phase = 0;
    bool failed = false;
    const int nl = a.L.nlast;

    for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        // ---- stage the tile: A[2c + q][j] = component q of x[j][c]
        if (GM == TC_DENSE) {
            const uint32_t c0 = (uint32_t)tile * 64u;
            for (int e = tid; e < 64 * kTcK; e += kTcThreads) {
                int c, j;
                if (a.inner == 1) { c = e >> 6; j = e & 63; }   // fibre contiguous
                else { j = e >> 6; c = e & 63; }                // columns contiguous
                float2 x = make_float2(0.f, 0.f);
                const uint32_t col = c0 + (uint32_t)c;
                if (j < nk && col < a.ncols) {
                    const uint32_t o = col / a.inner, in = col - o * a.inner;
                    x = a.in[((size_t)o * nk + j) * a.inner + in];
                }
                const float hr = tc_tf32(x.x), hi_ = tc_tf32(x.y);
                *reinterpret_cast<float*>(smem + S::A_hi + tc_off(2 * c, j)) = hr;
                *reinterpret_cast<float*>(smem + S::A_hi + tc_off(2 * c + 1, j)) = hi_;
                *reinterpret_cast<float*>(smem + S::A_lo + tc_off(2 * c, j)) = tc_tf32(x.x - hr);
                *reinterpret_cast<float*>(smem + S::A_lo + tc_off(2 * c + 1, j)) = tc_tf32(x.y - hi_);
            }
        } else {
            // row patterns and starts of the tile's 64 rows (fibre rows j, or active rows c)
            if (tid < 64) {
                uint64_t b = 0;
                uint32_t st = 0;
                if (GM == TC_FIBRE) {
                    const uint32_t r0 = a.units[tile];
                    const uint32_t rsk = a.L.rstride[a.mode];
                    const int i0 = (int)((r0 / rsk) % (uint32_t)nk);
                    if (tid >= i0 && tid < nk) {
                        const uint32_t r = r0 + (uint32_t)(tid - i0) * rsk;
                        b = row_bits(a.bits, r, nl);
                        if (b) st = rank_of(a.bits, a.off, (uint64_t)r * nl);
                    }
                } else {
                    const int64_t u = tile * 64 + tid;
                    if (u < *a.nunits) {
                        const uint32_t r = a.units[u];
                        b = row_bits(a.bits, r, nl);
                        st = rank_of(a.bits, a.off, (uint64_t)r * nl);
                    }
                }
                rb[tid] = b;
                rs[tid] = st;
            }
            __syncthreads();
            for (int e = tid; e < 64 * kTcK; e += kTcThreads) {
                int c, j;
                float2 x = make_float2(0.f, 0.f);
                if (GM == TC_FIBRE) {   // c = last-mode index, j = fibre row
                    j = e >> 6;
                    c = e & 63;
                    const uint64_t b = rb[j];
                    if (c < nl && ((b >> c) & 1ull))
                        x = a.in[rs[j] + (uint32_t)__popcll(b & ((1ull << c) - 1ull))];
                } else {                // c = row slot, j = last-mode index
                    c = e >> 6;
                    j = e & 63;
                    const uint64_t b = rb[c];
                    if (j < nl && ((b >> j) & 1ull))
                        x = a.in[rs[c] + (uint32_t)__popcll(b & ((1ull << j) - 1ull))];
                }
                x.x *= scale;
                x.y *= scale;
                const float hr = tc_tf32(x.x), hi_ = tc_tf32(x.y);
                *reinterpret_cast<float*>(smem + S::A_hi + tc_off(2 * c, j)) = hr;
                *reinterpret_cast<float*>(smem + S::A_hi + tc_off(2 * c + 1, j)) = hi_;
                *reinterpret_cast<float*>(smem + S::A_lo + tc_off(2 * c, j)) = tc_tf32(x.x - hr);
                *reinterpret_cast<float*>(smem + S::A_lo + tc_off(2 * c + 1, j)) = tc_tf32(x.y - hi_);
            }
        }
        // generic-proxy writes of the operands -> visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ah = tc_smem(smem + S::A_hi), al = tc_smem(smem + S::A_lo);
            const uint32_t bh = tc_smem(smem + S::B_hi), bl = tc_smem(smem + S::B_lo);
#pragma unroll
            for (int kk = 0; kk < kTcK / 8; ++kk) {
                const uint32_t ko = (uint32_t)kk * 2u * kTcLBO;   // 8 TF32 = two core matrices
                tc_mma(tmem, tc_desc(ah + ko), tc_desc(bh + ko), idesc, kk > 0);
                tc_mma(tmem + N, tc_desc(ah + ko), tc_desc(bl + ko), idesc, kk > 0);
                tc_mma(tmem + N, tc_desc(al + ko), tc_desc(bh + ko), idesc, 1);
            }
            tc_commit(mbar);
        }
        // ---- wait for the products (bounded)
        {
            const long long t0 = clock64();
            while (!tc_try_wait(mbar, phase)) {
                if (clock64() - t0 > kTcWaitCycles) {
                    failed = true;
                    break;
                }
            }
            phase ^= 1u;
        }
        failed = __syncthreads_or(failed) != 0;   // one decision for the whole CTA
        if (failed) {
            if (a.cnt) atomicOr(reinterpret_cast<unsigned long long*>(a.cnt + CNT_ERR), 4ull);
            break;
        }
        tc_fence_after();
        // ---- epilogue: this thread's TMEM lane is A row 2c + q
        const int c = tid >> 1, q = tid & 1;
        float* outf = reinterpret_cast<float*>(a.out);
#pragma unroll 1
        for (int ch = 0; ch < 4; ++ch) {   // outputs l = 16 ch .. 16 ch + 15
            float y[16], t[16];
            tc_ld16(tlane + 16 * ch, y);
            tc_ld16(tlane + N + 16 * ch, t);
#pragma unroll
            for (int i = 0; i < 16; ++i) y[i] += t[i];
            if (NMAT == 2) {   // complex matrix: combine with the partner lane's imaginary-part sums
                float di[16], dt[16];
                tc_ld16(tlane + 64 + 16 * ch, di);
                tc_ld16(tlane + N + 64 + 16 * ch, dt);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float mine = di[i] + dt[i];
                    const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
                    y[i] = q ? y[i] + other : y[i] - other;
                }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int l = 16 * ch + i;
                if (l >= nk) continue;
                if (GM == TC_DENSE) {
                    const uint32_t col = (uint32_t)tile * 64u + (uint32_t)c;
                    if (col >= a.ncols) continue;
                    const uint32_t o = col / a.inner, in = col - o * a.inner;
                    float* p = outf + 2 * (((size_t)o * nk + l) * a.inner + in) + q;
                    const float v = a.coef * y[i];
                    *p = a.accumulate ? *p + v : v;
                } else {
                    uint64_t b;
                    uint32_t pos;
                    bool act;
                    if (GM == TC_FIBRE) {   // output (row l, last-mode c)
                        b = rb[l];
                        act = c < nl && ((b >> c) & 1ull);
                        pos = rs[l] + (uint32_t)__popcll(b & ((1ull << c) - 1ull));
                    } else {                // output (row slot c, last-mode l)
                        b = rb[c];
                        act = l < nl && ((b >> l) & 1ull);
                        pos = rs[c] + (uint32_t)__popcll(b & ((1ull << l) - 1ull));
                    }
                    if (act) {
                        float* p = outf + 2 * (size_t)pos + q;
                        const float v = a.coef * y[i];
                        *p = a.accumulate ? *p + v : v;
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();   // TMEM and the operand tiles are reused by the next tile
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kCols)
                     : "memory");
    }
}

// ------------------------------------------------------------------ host
template <int NMAT, int GM>
static pq_status tc_launch(const TcArgs& a, int64_t grid_hint, cudaStream_t st) {
    using S = TcSmem<NMAT>;
    static bool attr = false;
    if (!attr) {
        PQ_CUDA_TRY(cudaFuncSetAttribute(k_tc_mode<NMAT, GM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::total));
        attr = true;
    }
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(grid_hint, grid_size()));
    k_tc_mode<NMAT, GM><<<G, kTcThreads, S::total, st>>>(a);
    PQ_CHECK_LAUNCH();
    return PQ_OK;
}

// Full grid (pvB): Y (+)= M along mode k of X, FP32.  M complex interleaved
// (row stride kMaxN); `real_only` applies its real part (the kinetic matrix).
pq_status tc_grid_mode(const State& s, const float2* X, float2* Y, const float* M, int k,
                       int accumulate, bool real_only, cudaStream_t st, const double* gate) {
    TcArgs a{};
    a.gate = gate;
    a.in = X;
    a.out = Y;
    a.M = M;
    a.mcomplex = 1;
    a.nk = s.lat.n[k];
    a.coef = 1.f;
    a.accumulate = accumulate;
    a.inner = s.lat.stride[k];
    a.ncols = s.lat.nfull / (uint32_t)a.nk;
    a.L = s.lat;
    a.cnt = s.cnt;
    const int64_t tiles = ((int64_t)a.ncols + 63) / 64;
    return real_only ? tc_launch<1, TC_DENSE>(a, tiles, st) : tc_launch<2, TC_DENSE>(a, tiles, st);
}

// Pruned set (pW): out (+)= coef P_A (M along mode k) in, FP32; M real (row
// stride kMaxN); in_scale / skip as for the other H.psi passes.
pq_status tc_pass(const State& s, const float2* in, float2* out, const float* M, int k, double coef,
                  int accumulate, const double* in_scale, const int* skip, int skip_k,
                  cudaStream_t st) {
    const Lattice& L = s.lat;
    TcArgs a{};
    a.in = in;
    a.out = out;
    a.M = M;
    a.mcomplex = 0;
    a.nk = L.n[k];
    a.coef = (float)coef;
    a.accumulate = accumulate;
    a.in_scale = in_scale;
    a.skip = skip;
    a.skip_k = skip_k;
    a.L = L;
    a.bits = s.bits;
    a.off = s.off;
    a.mode = k;
    a.cnt = s.cnt;
    const int64_t hint = (int64_t)grid_size();
    if (k == L.D - 1) {
        a.units = s.rows;
        a.nunits = s.cnt + CNT_ROWS;
        return tc_launch<1, TC_ROWS>(a, hint, st);
    }
    a.units = s.leaders + (size_t)k * s.rows_cap;
    a.nunits = s.cnt + CNT_LEAD0 + k;
    return tc_launch<1, TC_FIBRE>(a, hint, st);
}

}  // namespace pq
