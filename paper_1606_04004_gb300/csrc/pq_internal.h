// Internal declarations shared by the host and device translation units of
// the pruned-dynamics library.  Not part of the public ABI (see prunedq.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/prunedq.h"

namespace pq {

constexpr int kMaxD = 8;        // modes (a virtual size-1 mode is added for D = 1)
constexpr int kMaxN = 256;      // points per mode (row stride of the per-mode tables)
constexpr int kMaxNTile = 64;   // points per mode of the shared-memory tiled kernels and phase-space bases
constexpr int kMaxTerms = 64;   // potential terms
constexpr int kMaxK = 32;       // Krylov dimension

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();
extern std::atomic<int64_t> g_launches;

#define PQ_CUDA_TRY(expr)                                                       \
    do {                                                                        \
        cudaError_t e_ = (expr);                                                \
        if (e_ != cudaSuccess) {                                                \
            ::pq::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,          \
                            cudaGetErrorString(e_));                            \
            return PQ_ECUDA;                                                    \
        }                                                                       \
    } while (0)

#define PQ_LAUNCHED() ::pq::g_launches.fetch_add(1, std::memory_order_relaxed)

#ifdef PQ_BOUNDS_CHECK
// self-checking build: every launch is followed by a synchronisation so that
// an execution error names the launch that caused it
#define PQ_LAUNCH_SYNC() cudaDeviceSynchronize()
#else
#define PQ_LAUNCH_SYNC() cudaSuccess
#endif

#define PQ_CHECK_LAUNCH()                                                       \
    do {                                                                        \
        PQ_LAUNCHED();                                                          \
        cudaError_t e_ = cudaGetLastError();                                    \
        if (e_ == cudaSuccess) e_ = PQ_LAUNCH_SYNC();                           \
        if (e_ != cudaSuccess) {                                                \
            ::pq::set_error("%s:%d launch: %s", __FILE__, __LINE__,             \
                            cudaGetErrorString(e_));                            \
            return PQ_ECUDA;                                                    \
        }                                                                       \
    } while (0)

// ------------------------------------------------------------- lattice
// Row-major direct-product lattice.  A "row" is a run along the last mode
// (all digits but the last fixed); a "plane" fixes all digits but the last
// two.  Bits of the active-set bitmap are in linear-index order, so row r
// occupies bits [r*nlast, (r+1)*nlast).
struct Lattice {
    int D;                      // modes (>= 2 after the virtual leading mode)
    int n[kMaxD];               // points per mode
    uint32_t stride[kMaxD];     // linear-index strides
    uint32_t rstride[kMaxD];    // row-index strides (stride / nlast), modes < D-1
    uint32_t pstride[kMaxD];    // plane-index strides (stride / (n[D-2] nlast)), modes < D-2
    uint32_t nfull;             // lattice size
    uint32_t nrows;             // nfull / nlast
    uint32_t nplanes;           // nfull / (n[D-2] * nlast)
    uint32_t nwords;            // 64-bit bitmap words
    int nlast;                  // n[D-1]
    // lattice axes used by the neighbour rule of the adaption
    int naxes;
    int axis_n[2 * kMaxD];
    uint32_t axis_stride[2 * kMaxD];
};

// ------------------------------------------------------------- basis
struct Basis {
    int D_user = 0;                       // modes the caller declared
    std::vector<pq_mode_desc> modes;      // caller's modes
    std::vector<std::vector<double>> x, w, T;  // per caller mode
    // SoP Hamiltonian (DVR form): per-mode kinetic scale and potential terms
    bool sop_set = false;
    std::vector<double> kin_scale;                 // per caller mode
    std::vector<double> pot_coef;                  // per potential term
    std::vector<std::vector<double>> pot_values;   // [term][mode*n_mode + i] (1 for identity)
    std::vector<uint32_t> pot_mask;                // [term] bit k set: mode k not identity
    // phase-space modes: W (pW coefficients -> DVR coefficients), empty for DVR modes
    std::vector<std::vector<double>> W;
    bool generic = false;                          // some mode is a phase-space basis
    // pvB modes: G, B = G^-dagger, S = B^dagger B (complex, interleaved), empty otherwise
    std::vector<std::vector<double>> Gc, Bc, Sc;
    bool pvb = false;                              // all modes are pvB
    // generic SoP: per term the factor kind and values per mode
    struct GTerm {
        double coef;
        std::vector<int> kind;
        std::vector<std::vector<double>> values;
    };
    std::vector<GTerm> gterms;
    // tabulated diagonal potential on the whole lattice (empty: none)
    std::vector<double> vgrid;
};

pq_status build_dvr_mode(const pq_mode_desc& m, std::vector<double>& x,
                         std::vector<double>& w, std::vector<double>& T);
pq_status build_pw_mode(const pq_mode_desc& m, std::vector<double>& x, std::vector<double>& w,
                        std::vector<double>& T, std::vector<double>& W);
pq_status build_pvb_mode(const pq_mode_desc& m, std::vector<double>& x, std::vector<double>& w,
                         std::vector<double>& T, std::vector<double>& G, std::vector<double>& B,
                         std::vector<double>& S);
// Normalised packet factors f_k(i) = sqrt(w_i) g_k(x_i) / ||.||, complex interleaved.
void packet_factors(const Basis& b, const double* q0, const double* p0, const double* width,
                    std::vector<double>& out /* D_int * kMaxN * 2 */, int lead_virtual);
int jacobi_eigh(int n, std::vector<double>& A, std::vector<double>& evals,
                std::vector<double>& evecs);

// ------------------------------------------------------------- state
struct Timing {
    bool enabled = false;
    double ms = 0;
    int64_t n_apply = 0;
    double coef = 0;
    std::vector<cudaEvent_t> ev_start, ev_stop;   // pairs per recorded apply
    std::vector<int64_t> ev_coef_slot;            // unused placeholder
};

struct ObsRecord {
    double t, c_re, c_im, norm2, energy;
    int64_t n_active, n_wasted;
};

// Device-side per-state counters (one int64 array).
enum Counter : int {
    CNT_NA = 0,        // active points
    CNT_ROWS = 1,      // active rows
    CNT_PLANES = 2,    // active planes
    CNT_ERR = 3,       // error bits (1: capacity overflow, 2: numeric)
    CNT_NA_OLD = 4,    // active points before the last rebuild
    CNT_EXCL = 5,      // adaption: members of A outside S + N(S)
    CNT_LEAD0 = 8,     // fibre leaders of outer mode k at CNT_LEAD0 + k
    CNT_FAULT = 24,    // bounds-check build: site, index, bound of the first bad access
    CNT_SIZE = 32
};

// Device scalars of the Krylov step (FP64).
struct KrylovScalars {
    double beta0;                 // ||psi||
    double sigma[kMaxK + 1];      // scale of stored Krylov vector k
    double alpha[kMaxK];
    double beta[kMaxK];
    double dots[2 * (kMaxK + 1)]; // <V_i, W> (re, im) of the current step
    double hnorm2;                // ||W||^2 before orthogonalisation
    double coef[2 * kMaxK];       // final combination coefficients (re, im)
    double renorm;                // FP32-mix: norm correction for the next step (0: none)
    double rn_target;             // FP32-mix: norm the step's output should have (0: unset)
    double rn_last;               // FP32-mix: norm of the last step's output
    int keff;                     // Krylov dimension reached (breakdown)
    int pad;
    double obs[8];                // C re, C im, norm2, wasted (as double)
};

struct State {
    const Basis* basis = nullptr;
    Lattice lat{};
    int prec = PQ_FP64;
    int lead_virtual = 0;          // 1 if a virtual size-1 leading mode was added
    size_t cap = 0;                // capacity (active points)
    size_t esize = 16;             // bytes per coefficient
    // device buffers
    uint32_t* keys = nullptr;      // sorted active linear indices
    void* psi = nullptr;           // coefficients
    void* psi_alt = nullptr;       // prune target / apply scratch
    uint64_t* bits = nullptr;      // active-set bitmap
    uint64_t* bits_alt = nullptr;
    uint32_t* off = nullptr;       // rank offsets (exclusive popcount prefix), nwords+1
    uint32_t* off_alt = nullptr;
    uint32_t* rows = nullptr;      // active row ids
    uint32_t* planes = nullptr;    // active plane ids
    uint32_t* leaders = nullptr;   // fibre leaders, (D-2) lists of nrows_cap entries
    uint2* rowinfo = nullptr;      // per lattice row: (position of its first active point,
                                   // active pattern); (0, 0) for empty rows.  Only when
                                   // n[D-1] <= 32 and the lattice has at most 2^28 rows.
    size_t rows_cap = 0;
    // FP32 H.psi path hint: 1 = dense-tile passes (at least half the lattice
    // active), 0 = item-blocked passes, -1 = unknown (both launched, the
    // device-side set size picks).  Either path is correct for any set; a
    // stale hint costs speed only.
    int dense_hint = -1;
    int64_t* h_na = nullptr;       // pinned: two lagged copies of the active-set size
    int64_t* cnt = nullptr;        // counters (CNT_*)
    uint32_t* scan_tmp = nullptr;  // block sums of the scans
    double* red_tmp = nullptr;     // block partials of the reductions
    KrylovScalars* ks = nullptr;   // device Krylov scalars
    void* V = nullptr;             // Krylov vectors, (K+1) * cap
    int V_K = 0;
    // Hamiltonian tables (device), both precisions
    double* T64 = nullptr;  float* T32 = nullptr;      // [D][kMaxN][kMaxN]
    double* pot64 = nullptr; float* pot32 = nullptr;   // [nterms][D][kMaxN]
    double* vgrid64 = nullptr; float* vgrid32 = nullptr;   // tabulated V on the lattice, or null
    int nterms = 0;
    int ngroup[4] = {0, 0, 0, 0};  // potential terms by the tile modes they touch (see apply_h.cu)
    // generic SoP (phase-space bases): dense 1D matrices and the pass plan
    bool generic = false;
    double* gmat64 = nullptr; float* gmat32 = nullptr;   // [nmat][kMaxN][kMaxN]
    int gsingle[kMaxD];            // merged single-mode matrix per mode (-1: none)
    struct GPass { int mode, mat; };
    struct GPlan { double coef; std::vector<GPass> passes; };   // passes: descending mode
    std::vector<GPlan> gplan;      // terms with two or more factors
    void* gtmp = nullptr;          // two scratch vectors (capacity each) for those terms
    // pvB (Sec. 2.2): complex per-mode matrices [D][kMaxN][kMaxN][2], full-grid
    // buffers (3 x lattice), 5 work vectors (capacity each), the packet's bra
    // factors B^dagger f (the coefficients use G^dagger f)
    bool pvb = false;
    double* pvbB64 = nullptr; float* pvbB32 = nullptr;
    double* pvbBh64 = nullptr; float* pvbBh32 = nullptr;
    double* pvbS64 = nullptr; float* pvbS32 = nullptr;
    double* pvbSi64 = nullptr; float* pvbSi32 = nullptr;   // S^-1 = G^dagger G (CG preconditioner)
    int pvb_cg_pred = 16;          // conjugate-gradient iterations launched before the first poll
    cudaStream_t cap_stream = nullptr;   // private stream the CG iteration is captured on
    double* pvbT64 = nullptr; float* pvbT32 = nullptr;
    void* pvb_grid = nullptr;
    void* pvb_vec = nullptr;
    double* fac_bra64 = nullptr;
    double pvb_smax = 1.0;
    double* fac64 = nullptr; float* fac32 = nullptr;   // packet factors [D][kMaxN] complex
    // host side
    double t = 0;
    std::vector<ObsRecord> obs;
    bool obs_energy_pending = false;
    double theta = 0;
    int radius = 1;
    Timing timing;
    int64_t* h_cnt = nullptr;      // pinned mirror of cnt
    double q0[kMaxD] = {0}, p0[kMaxD] = {0}, width[kMaxD] = {0};   // packet (caller modes)
    void* io_in = nullptr;         // staging buffers of pq_apply_H_host
    void* io_out = nullptr;
    cudaStream_t last_stream = nullptr;
};

// lattice.cu
pq_status lattice_setup(State& s);
pq_status rebuild_from_bits(State& s, bool remap, cudaStream_t st);
// Neighbour rules (pq_neighbour_rule) and the relative exclusion threshold
// of the adaption; radius 2 (the full box) needs at most kMaxBoxAxes axes.
constexpr int kMaxBoxAxes = 8;
// Device memory through the caller's allocator when one is set
// (pq_set_allocator), else cudaMalloc / cudaMallocAsync (`async`: stream-ordered).
void* dev_alloc(size_t bytes, cudaStream_t st, bool async);
void dev_free(void* p, cudaStream_t st, bool async);
pq_status check_neighbour_rule(const Lattice& L, int radius);
pq_status prune_launch(State& s, double theta, int radius, double rel_excl, cudaStream_t st);
pq_status init_bits_from_packet(State& s, double theta, cudaStream_t st);
pq_status set_psi_from_packet(State& s, cudaStream_t st);
// FP32-mix norm keeping (see krylov.cu): forget the target norm and the pending
// correction (the coefficients were replaced)
pq_status reset_norm_keeping(State& s, cudaStream_t st);
// Replace the active set by n sorted keys on the device; with remap the
// current coefficients are carried over (kept where the point stays, zero
// where it is new), else they are left undefined.
pq_status load_set(State& s, const uint32_t* d_keys, int64_t n, cudaStream_t st,
                   bool remap = false);
int grid_size();

// tc_fibre.cu: dense 1D operators on the tensor cores (FP32 data, split TF32)
// Full grid: Y (+)= M along mode k of X (M complex interleaved, or its real part).
// `gate` (device, nullable): the launch does nothing while *gate != 0.
pq_status tc_grid_mode(const State& s, const float2* X, float2* Y, const float* M, int k,
                       int accumulate, bool real_only, cudaStream_t st,
                       const double* gate = nullptr);
// Pruned set: out (+)= coef P_A (M along mode k) in, M real.
pq_status tc_pass(const State& s, const float2* in, float2* out, const float* M, int k, double coef,
                  int accumulate, const double* in_scale, const int* skip, int skip_k,
                  cudaStream_t st);
constexpr int kTcMaxN = 64;   // matrix size and last-mode length the tensor-core passes take

// apply_h.cu
// in_scale (device, nullable): the input is multiplied by *in_scale on load.
// skip (device, nullable): the launch does nothing when *skip <= skip_k.
pq_status apply_H_launch(const State& s, const void* in, void* out, int prec,
                         const double* in_scale, const int* skip, int skip_k,
                         cudaStream_t st);

// krylov.cu
pq_status propagate_impl(State& s, const pq_prop_desc& d, int nsteps, cudaStream_t st);
pq_status ensure_krylov(State& s, int K);
// One SIL step of the state's coefficients on the current set (no adaption,
// no observables); dt may be negative (backward propagation).
pq_status sil_only(State& s, const pq_prop_desc& d, cudaStream_t st);
pq_status observe_launch(State& s, double theta, cudaStream_t st);
pq_status energy_of_current(State& s, double* E, cudaStream_t st);

// pvb.cu
pq_status pvb_apply(State& s, const void* in, void* out, int prec, cudaStream_t st);
pq_status pvb_observe_current(State& s, double theta, cudaStream_t st);
pq_status pvb_propagate(State& s, const pq_prop_desc& d, int nsteps, cudaStream_t st);

// capi.cu: an FP64 state on the basis, capacity and packet of s (empty set),
// and its release
pq_status make_fp64_twin(const State& s, State** out);
void free_twin(State* t);

// adjoint.cu
pq_status survival_grad(State& s, const pq_prop_desc& d, int nsteps, int ckpt,
                        const pq_param_desc* params, int np, double* grad, double* P_out,
                        cudaStream_t st);

}  // namespace pq
