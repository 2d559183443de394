// Observables of the current state without any device allocation.
//
// Some callers cannot let a library call cudaMalloc / cudaFree between
// steps: code that runs under a framework whose allocator owns the whole
// device-memory budget, or loops that must not trigger the device-wide
// synchronisation an allocation or a free implies.  pq_observe_noalloc serves
// them: it computes the same quantities as the observables the propagation
// records (C(t), ||psi||^2, the number of small coefficients), keeping its
// per-block partial sums in a fixed file-scope device array instead of
// allocated scratch.
#include <mutex>

#include "device_util.cuh"

namespace pq {

// Fixed scratch: kNoAllocMaxBlocks blocks x 4 partial sums, then a 4-double
// result.  Every GPU that loads the library holds this 1 MiB until exit.
constexpr int kNoAllocChunk = 8192;          // active points per block
constexpr int kNoAllocMaxBlocks = 32768;     // -> at most 268,435,456 active points
constexpr int kNoAllocThreads = 256;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks * 4 + 4];

// Symbol address per device, taken once with that device current.
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {nullptr};

static pq_status noalloc_scratch(double** out) {
    int dev = 0;
    PQ_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return PQ_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error("cudaGetSymbolAddress of the fixed scratch failed: %s",
                      cudaGetErrorString(e));
            return PQ_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return PQ_OK;
}

// Block b reduces active points [b*chunk, (b+1)*chunk) into partials[b][0..3]:
// C re, C im (C = sum conj(a0_I) psi_I), ||psi||^2, count of |a| < theta.
template <typename R>
__global__ void __launch_bounds__(kNoAllocThreads)
k_observe_chunks(const uint32_t* __restrict__ keys, const typename Cx<R>::T* __restrict__ psi,
                 int64_t n, Lattice L, const typename Cx<R>::T* __restrict__ fac, double theta2,
                 float lo, float hi, double* partials) {
    const int64_t start = (int64_t)blockIdx.x * kNoAllocChunk;
    const int64_t end = min(n, start + kNoAllocChunk);
    double cr = 0.0, ci = 0.0, nn = 0.0, wasted = 0.0;
    for (int64_t p = start + threadIdx.x; p < end; p += blockDim.x) {
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
        cr += (double)(ar * v.x + ai * v.y);
        ci += (double)(ar * v.y - ai * v.x);
        nn += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        bool sig;
        if (sizeof(R) == 8)
            sig = significant64((double)v.x, (double)v.y, theta2);
        else
            sig = significant32((float)v.x, (float)v.y, theta2, lo, hi);
        if (!sig) wasted += 1.0;
    }
    __shared__ double sh[4][kNoAllocThreads / 32];
    double vals[4] = {cr, ci, nn, wasted};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < 4; ++j) {
        const double v = warp_sum(vals[j]);
        if (lane == 0) sh[j][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0.0;
        for (int w = 0; w < kNoAllocThreads / 32; ++w) acc += sh[threadIdx.x][w];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = acc;
    }
}

// result[j] = sum over blocks (in block order) of partials[b][j]
__global__ void k_observe_chunks_done(const double* partials, int nblocks, double* result) {
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j >= 4) return;
    double acc = 0.0;
    for (int b = lane; b < nblocks; b += 32) acc += partials[(size_t)b * 4 + j];
    acc = warp_sum(acc);
    if (lane == 0) result[j] = acc;
}

}  // namespace pq

using namespace pq;

extern "C" __attribute__((visibility("default"))) pq_status pq_observe_noalloc(
    const pq_state* state, double theta, double* out, void* stream) {
    clear_error();
    const State* s = reinterpret_cast<const State*>(state);
    if (!s || !out || !(theta >= 0)) {
        set_error("null state or output, or theta < 0");
        return PQ_EINVAL;
    }
    if (s->pvb) {
        // pvB needs the bra factors B^dagger f and the norm a^dagger S_AA a
        // (Sec. 2.2), which take full-grid transforms and their buffers
        set_error("pq_observe_noalloc does not provide pvB states; use pq_observables_get");
        return PQ_ENOTSUP;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* scratch = nullptr;
    pq_status rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    int64_t hc[CNT_SIZE];
    PQ_CUDA_TRY(cudaMemcpyAsync(hc, s->cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    PQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (hc[CNT_ERR] & 1) {
        set_error("the state's active set outgrew its capacity");
        return PQ_ECAPACITY;
    }
    const int64_t n = hc[CNT_NA];
    const int64_t nblocks = (n + kNoAllocChunk - 1) / kNoAllocChunk;
    if (nblocks > kNoAllocMaxBlocks) {
        set_error("pq_observe_noalloc supports at most %lld active points (%lld given)",
                  (long long)kNoAllocMaxBlocks * kNoAllocChunk, (long long)n);
        return PQ_EINVAL;
    }
    double* partials = scratch;
    double* result = scratch + (size_t)kNoAllocMaxBlocks * 4;
    // the result must start from zero when the set is empty (no block runs)
    PQ_CUDA_TRY(cudaMemsetAsync(result, 0, 4 * sizeof(double), st));
    const double theta2 = theta * theta;
    float lo = -1.0f, hi = 3.0e38f;
    if (theta2 >= 1e-30) {
        lo = (float)(theta2 * (1.0 - 1e-5));
        hi = (float)(theta2 * (1.0 + 1e-5));
    }
    if (nblocks > 0) {
        if (s->prec == PQ_FP64)
            k_observe_chunks<double><<<(unsigned)nblocks, kNoAllocThreads, 0, st>>>(
                s->keys, (const double2*)s->psi, n, s->lat, (const double2*)s->fac64, theta2,
                lo, hi, partials);
        else
            k_observe_chunks<float><<<(unsigned)nblocks, kNoAllocThreads, 0, st>>>(
                s->keys, (const float2*)s->psi, n, s->lat, (const float2*)s->fac32, theta2, lo,
                hi, partials);
        PQ_CHECK_LAUNCH();
        k_observe_chunks_done<<<1, 128, 0, st>>>(partials, (int)nblocks, result);
        PQ_CHECK_LAUNCH();
    }
    double h[4];
    PQ_CUDA_TRY(cudaMemcpyAsync(h, result, sizeof(h), cudaMemcpyDeviceToHost, st));
    PQ_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < 4; ++j) out[j] = h[j];
    return PQ_OK;
}
