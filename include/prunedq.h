/*
 * prunedq.h -- C ABI of the GB300 (sm_103a) pruned quantum-dynamics library.
 *
 * The library propagates a wavepacket that lives only on an active, non
 * direct-product subset A of a direct-product basis (Larsson, Hartke, Tannor,
 * arXiv:1606.04004).  A sum-of-products (SoP) Hamiltonian acts along the
 * partial fibres of A (Sec. 2.2.2, Appendix), inside short-iterative-Lanczos
 * steps (Sec. 3.1), and after each step a threshold prune plus a
 * nearest-neighbour add rebuilds A (Sec. 2.5).
 *
 * Conventions shared by every call:
 *  - Every call returns a pq_status; PQ_OK is 0.  No C++ exception crosses
 *    the ABI.  pq_last_error() gives a message for the last failing call of
 *    the calling thread.
 *  - A lattice point is named by its row-major linear index (mode 0 slowest,
 *    mode D-1 contiguous).  A is kept sorted by that index.  The product of
 *    the mode sizes must be below 2^32 and every mode size at most 256
 *    (modes of up to 64 points take the tiled H.psi kernels, longer modes
 *    the point-parallel ones).
 *  - Coefficient vectors are complex, interleaved (re, im): double pairs for
 *    PQ_FP64, float pairs for PQ_FP32MIX.  Vectors passed to the library as
 *    "device" pointers live in device memory of the current CUDA device and
 *    stay owned by the caller; the library never frees them.
 *  - `stream` is a cudaStream_t handle passed as void*; NULL means the
 *    legacy default stream.  Calls that take a stream enqueue their work on
 *    it and return without synchronising unless stated.
 *  - Objects (pq_basis, pq_state) are owned by the library; free them with
 *    the matching *_free call.  They are not thread-safe: one host thread
 *    (and one stream) at a time per object.
 */
#ifndef PRUNEDQ_H
#define PRUNEDQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pq_status {
    PQ_OK = 0,
    PQ_EINVAL = 1,      /* bad argument (shape, size, range, null pointer)   */
    PQ_ENOMEM = 2,      /* host or device allocation failed                   */
    PQ_ECUDA = 3,       /* a CUDA runtime call failed                         */
    PQ_ECAPACITY = 4,   /* the active set outgrew the state's capacity        */
    PQ_ENUMERIC = 5,    /* NaN / Inf met in a norm or Lanczos coefficient     */
    PQ_ETIMEOUT = 6,    /* a bounded device wait ran out                      */
    PQ_EBREAKDOWN = 7,  /* Lanczos breakdown where it is not allowed          */
    PQ_ENOTSUP = 8      /* valid request that the library does not implement */
} pq_status;

typedef enum pq_basis_kind {
    PQ_SINE_DVR = 0,  /* sine DVR on a box (Sec. 2.2: admissible non-periodic DVR) */
    PQ_HO_DVR = 1,    /* harmonic-oscillator (Gauss-Hermite) DVR (Sec. 3.3)       */
    PQ_PVB = 2,       /* biorthogonal projected von Neumann basis (Sec. 2.2)      */
    PQ_PW = 3,        /* projected Weylets (Sec. 2.4)                             */
    PQ_FGH_DVR = 4    /* Fourier grid DVR on a periodic box (Sec. 2.2, Sec. 3.1)  */
} pq_basis_kind;

typedef enum pq_precision {
    PQ_FP64 = 0,      /* complex FP64 storage and arithmetic                      */
    PQ_FP32MIX = 1    /* complex FP32 H.psi, FP64 Lanczos scalars, norms and sums */
} pq_precision;

/* Neighbour rules of the adaption (Sec. 3.1, "phase-space ball radius"), on
 * the lattice axes: one per DVR mode, two (x and p) per phase-space mode.
 * An interior point on k axes gets 2k, 2k^2 or 3^k - 1 neighbours; points
 * outside the lattice are dropped.  PQ_RADIUS_2 is limited to 8 axes. */
typedef enum pq_neighbour_rule {
    PQ_RADIUS_1 = 1,      /* +-1 along one axis                                  */
    PQ_RADIUS_SQRT2 = 2,  /* +-1 along one axis or along two axes at once        */
    PQ_RADIUS_2 = 3       /* every offset in {-1, 0, +1}^k except 0              */
} pq_neighbour_rule;

/* One mode of the direct-product basis.
 *  kind   pq_basis_kind.
 *  n      number of points (2..256).  Lattices
 *         with a mode longer than 64 use a point-parallel H.psi meant for
 *         small lattices (the 2D FGH double well).
 *  xmin, xmax  box edges: sine DVR points at xmin + j L/(n+1), j=1..n; FGH
 *         points at xmin + j L/n, j=0..n-1 on the periodic box [xmin, xmax).
 *  mass   mass in the kinetic energy -d^2/dx^2 / (2 mass).
 *  omega  frequency of the HO-DVR's underlying oscillator (with `mass`).
 *  nx_lattice, np_lattice  phase-space lattice of pvB / pW modes (unused for DVRs).
 *  dvr    underlying DVR of a pvB / pW mode: PQ_SINE_DVR (0, default) or
 *         PQ_FGH_DVR (Sec. 3.1 builds both phase-space bases on the FGH grid).
 */
typedef struct pq_mode_desc {
    int kind;
    int n;
    double xmin, xmax;
    double mass;
    double omega;
    int nx_lattice, np_lattice;
    int dvr;
} pq_mode_desc;

typedef struct pq_basis pq_basis;
typedef struct pq_state pq_state;

/* Build the per-mode 1D bases (Sec. 2.1 direct-product expansion; DVR grid
 * points x_j, weights w_j with a_j = sqrt(w_j) psi(x_j), and kinetic matrices).
 * Host-only FP64 work.  *out is owned by the library: free with pq_basis_free.
 * Errors: PQ_EINVAL for D outside 1..7, n outside 2..256, a lattice of 2^32
 * points or more, or an unknown kind; PQ_ENOTSUP for pvB modes mixed with
 * other kinds. */
pq_status pq_build_basis(const pq_mode_desc* modes, int D, pq_basis** out);
void pq_basis_free(pq_basis* basis);

/* Copy mode `mode`'s grid points and weights (n doubles each; either pointer
 * may be NULL) or its kinetic matrix (n*n doubles, row-major) to host memory. */
pq_status pq_basis_grid(const pq_basis* basis, int mode, double* x, double* w);
pq_status pq_basis_kinetic(const pq_basis* basis, int mode, double* T);

/* Mode `mode`'s transformation from basis coefficients to DVR coefficients
 * (n*n doubles, row-major, a^chi = W a): the projected Weylets' W = Phi S^(-1/2)
 * (Sec. 2.4); the unit matrix for a DVR mode. */
pq_status pq_basis_transform(const pq_basis* basis, int mode, double* W);

/* Sum-of-products Hamiltonian H = sum_l coef_l (x)_kappa h^(kappa,l)
 * (Sec. 2.2.2).  Each term gives one factor per mode:
 *   PQ_FACTOR_IDENTITY  the unit matrix;
 *   PQ_FACTOR_KINETIC   the mode's kinetic matrix;
 *   PQ_FACTOR_DIAG      a diagonal (potential) factor given by its n values
 *                       at the DVR points (copied).
 * In a DVR basis the potential is diagonal (Sec. 2.1), so a term is either
 * kinetic (one KINETIC factor, IDENTITY elsewhere) or potential (only DIAG /
 * IDENTITY factors).  Other combinations return PQ_ENOTSUP.  At most 64
 * potential terms.  Replaces any previous SoP of the basis. */
typedef enum pq_factor_kind {
    PQ_FACTOR_IDENTITY = 0,
    PQ_FACTOR_KINETIC = 1,
    PQ_FACTOR_DIAG = 2
} pq_factor_kind;

typedef struct pq_factor {
    int kind;              /* pq_factor_kind                               */
    const double* values;  /* n values for PQ_FACTOR_DIAG, else ignored     */
} pq_factor;

typedef struct pq_sop_term {
    double coef;
    const pq_factor* factors;  /* D entries, one per mode                  */
} pq_sop_term;

pq_status pq_set_sop(pq_basis* basis, const pq_sop_term* terms, int nterms);

/* A diagonal potential given as a table over the whole lattice (not in SoP
 * form; Sec. 2.1: in a DVR the potential is diagonal, V_II = V(x_I)), added to
 * the SoP potential: n values, row-major over the modes (the last mode
 * fastest), copied.  States created afterwards use it.  V = NULL removes it.
 * Errors: PQ_EINVAL (n is not the lattice size, a value not finite),
 * PQ_ENOTSUP (pW or pvB bases). */
pq_status pq_set_potential_grid(pq_basis* basis, const double* V, int64_t n);

/* Create a state holding a product Gaussian packet
 *   psi(q) = prod_k (2 pi w_k^2)^(-1/4) exp(-(q_k-q0_k)^2/(4 w_k^2) + i p0_k (q_k-q0_k))
 * projected on the DVR (a_I = prod_k sqrt(w_{i_k}) psi_k(x_{i_k}), each mode
 * normalised, so ||a|| = 1 on the full lattice), followed by the initial
 * adaption of Sec. 2.5 with threshold `theta` and neighbour rule `radius`
 * (pq_neighbour_rule).  q0, p0, width: D doubles each (host).  `capacity` is the
 * largest active-set size the state can hold (0 = the full lattice); device
 * memory for the Krylov space is taken when pq_propagate first needs it.
 * The state keeps the normalised full-lattice packet (as its D factors) as
 * Psi(0) for the autocorrelation.  The basis must outlive the state.
 * Synchronises the device.  Errors: PQ_EINVAL, PQ_ENOMEM, PQ_ECAPACITY. */
pq_status pq_init_packet(const pq_basis* basis, const double* q0, const double* p0,
                         const double* width, double theta, int radius, int precision,
                         size_t capacity, pq_state** out);
void pq_state_free(pq_state* state);

/* Replace the state's active set and coefficients (host arrays): `idx` holds
 * n sorted, distinct linear indices, `psi` n complex values of the state's
 * precision (may be NULL: zeros).  Synchronises.  PQ_EINVAL if idx is not
 * strictly increasing or out of the lattice, PQ_ECAPACITY if n > capacity. */
pq_status pq_state_load(pq_state* state, const int64_t* idx, int64_t n, const void* psi);

/* Number of active points (synchronises the device). */
pq_status pq_state_size(const pq_state* state, int64_t* n_active);

/* Copy the active set (n_active int64 linear indices) and / or the
 * coefficients (n_active complex values of the state's precision) to host
 * memory; either pointer may be NULL.  Synchronises. */
pq_status pq_state_read(const pq_state* state, int64_t* idx, void* psi);

/* Device address of the state's coefficient vector (valid until the next
 * call that changes the active set). */
pq_status pq_state_psi_device(const pq_state* state, void** psi);

/* Pruned H.psi on the state's current active set (Sec. 2.2.2 pruned
 * sequential transform; Appendix, fibre transform over one mode at a time):
 *   out_I = sum_kappa sum_{j : I[kappa->j] in A} T^kappa_{i_kappa j} in_{I[kappa->j]}
 *           + V(x_I) in_I,     I in A,
 * which equals P_A H P_A in for a DVR Hamiltonian (diagonal V, Sec. 2.1).
 * in, out: device arrays of n_active complex values in A's order, of the type
 * `precision` selects (it may differ from the state's own precision); they
 * must not overlap.  out_vHv (nullable): device address of two doubles that
 * receive Re and Im of <in, out> = sum_I conj(in_I) out_I (the Lanczos
 * alpha of a normalised `in`, Sec. 3.1), summed in FP64 in a fixed order; it
 * uses the state's reduction scratch, so calls on one state must not overlap
 * on the device.  No allocation.  Asynchronous on `stream`.  */
pq_status pq_apply_H(const pq_state* state, const void* in, void* out, int precision,
                     double* out_vHv, void* stream);

/* Same operator with host buffers: copies `in` (host, n_active complex of
 * `precision`) to the device, applies H, copies the result to `out` (host)
 * and synchronises `stream`.  Uses the state's own device buffers. */
pq_status pq_apply_H_host(pq_state* state, const void* in, void* out, int precision,
                          void* stream);

/* Adaption of Sec. 2.5 on the state's current coefficients: S = {I in A :
 * |a_I| >= theta} (tested as fl(re*re) + fl(im*im) >= fl(theta*theta) in
 * FP64, FP32 values widened exactly), A' = S union (nearest neighbours of S
 * of the rule `radius`, pq_neighbour_rule, clipped at the edges); kept
 * coefficients are carried over, new ones are zero.  Relative exclusion
 * (Sec. 2.5: functions leave only when their number exceeds a threshold
 * relative to the set): when at most rel_excl * |A| members of A fall outside
 * A', all of A stays (rel_excl = 0: no such rule).  Asynchronous; a capacity
 * overflow is reported by the next synchronising call as PQ_ECAPACITY.
 * Errors: PQ_EINVAL (theta or rel_excl negative or not finite, unknown rule),
 * PQ_ENOTSUP (PQ_RADIUS_2 on more than 8 lattice axes). */
pq_status pq_prune(pq_state* state, double theta, int radius, double rel_excl, void* stream);

/* Propagation (Sec. 3.1): per step, a short-iterative-Lanczos step of order K
 * with time step dt (each new Krylov vector orthogonalised against all
 * previous ones when reorth = 1, against the previous two when reorth = 0;
 * FP64 Lanczos scalars), then the adaption with (theta, radius, rel_excl), then the
 * observables of the new state: t, C(t) = <Psi(0)|Psi(t)>, ||psi||^2,
 * E = Re<psi|H psi>/||psi||^2, |A|, and the number of active points with
 * |a| < theta.  Observables accumulate in the state (pq_observables_get).
 * PQ_FP32MIX states: the SIL step keeps the norm in exact arithmetic, so the
 * run carries in FP64 the norm each step's output should have (following the
 * adaption) and folds the correction into the next step's combination
 * coefficients; FP32 rounding then no longer adds up into a norm drift.
 * Asynchronous except for one synchronisation at the start and one at the
 * end that reads the device error word (and non-blocking reads of the set
 * size that choose between two H.psi paths, equal up to rounding). */
typedef struct pq_prop_desc {
    int K;           /* Krylov dimension (H.psi products per step), 1..32     */
    double dt;       /* time step                                            */
    double theta;    /* adaption threshold                                    */
    int radius;      /* neighbour rule of the adaption (pq_neighbour_rule)    */
    int reorth;      /* 1 = full re-orthogonalisation, 0 = three-term         */
    double rel_excl; /* relative exclusion threshold of the adaption (0: none) */
    int integrator;  /* pq_integrator: PQ_SIL (order K) or PQ_RK4             */
    double sil_tol;  /* SIL only: > 0 makes the order error-controlled, up to K:
                        a step stops after k + 1 vectors once
                        beta_k |[exp(-i T_{k+1} dt) e_1]_k| <= sil_tol         */
} pq_prop_desc;

/* Time steppers of pq_propagate.  PQ_RK4 is the classical fourth-order
 * Runge-Kutta step (four H.psi per step; not in the paper, whose propagator
 * is SIL, Sec. 3.1); it is not norm-conserving and needs dt ||H|| < 2.8.
 * Not provided for pvB states or by pq_survival_grad (PQ_ENOTSUP). */
typedef enum pq_integrator { PQ_SIL = 0, PQ_RK4 = 1 } pq_integrator;

pq_status pq_propagate(pq_state* state, const pq_prop_desc* desc, int nsteps, void* stream);

/* Observables recorded so far, oldest first (index 0 = after the initial
 * prune, t = 0).  The caller passes arrays of `capacity` entries (any may be
 * NULL); *count receives the number of records (copied: min(count, capacity)).
 * E of the newest record needs one more H.psi and is computed here. */
typedef struct pq_observables {
    int64_t capacity;
    int64_t* count;
    double* t;
    double* c_re;
    double* c_im;
    double* norm2;
    double* energy;
    int64_t* n_active;
    int64_t* n_wasted;
} pq_observables;

pq_status pq_observables_get(pq_state* state, pq_observables* out);

/* Time spent in pq_apply_H-equivalent work inside pq_propagate, measured with
 * CUDA events on the propagation stream while timing is enabled: total
 * milliseconds, number of H.psi products and the summed active-set size over
 * those products.  pq_set_timing(state, 1) enables and resets it. */
pq_status pq_set_timing(pq_state* state, int enable);
pq_status pq_timing_get(pq_state* state, double* apply_ms, int64_t* n_apply,
                        double* coef_applied);

/* Gradient of the survival probability P = |<Psi(0)|Psi(T)>|^2 (Psi(0) the
 * normalised full packet, as in the autocorrelation of Eq. acorr), T =
 * nsteps * desc->dt, with respect to parameters of the Hamiltonian or of the
 * packet.  The paper computes C(t) only; the gradient is taken of that
 * quantity.  The run starts from the state's initial packet and adaption;
 * the sequence of active sets of that run is recorded and then held fixed
 * (the map is differentiable only with the sets frozen).  The gradient is
 * that of the discrete propagation: a reverse sweep through every SIL step
 * (its Lanczos recurrence repeated in FP64 and run backwards, the derivative
 * of the tridiagonal exponential in its eigenbasis), psi_n recomputed from
 * checkpoints taken every `ckpt_every` steps, so it agrees with finite
 * differences of the propagation whether or not the step has converged.
 * Precision: the forward run (sets, C, P) in the state's precision; for a
 * PQ_FP32MIX state an internal FP64 copy of the state replays the run on its
 * recorded sets for the checkpoints, and the reverse sweep is FP64.
 * Errors: PQ_ENUMERIC for a non-finite Lanczos scalar or gradient.
 * Parameters:
 *   PQ_PARAM_POTENTIAL  dH/dtheta as diagonal SoP terms on the DVR grid
 *                       (PQ_FACTOR_DIAG / PQ_FACTOR_IDENTITY factors);
 *   PQ_PARAM_CENTRE     the packet centre q0 of `mode`.
 * grad_out: nparams doubles (host); P_out (nullable): P.  DVR bases and
 * fixed-order SIL only (PQ_ENOTSUP otherwise: pW / pvB, PQ_RK4, sil_tol > 0),
 * at most 16 parameters.  The state is left at its
 * initial packet; its recorded observables are not changed.  Synchronises.
 * Allocates device memory for the recorded sets and checkpoints. */
typedef enum pq_param_kind { PQ_PARAM_POTENTIAL = 0, PQ_PARAM_CENTRE = 1 } pq_param_kind;

typedef struct pq_param_desc {
    int kind;                   /* pq_param_kind                                  */
    int mode;                   /* PQ_PARAM_CENTRE: mode whose q0 is the parameter */
    const pq_sop_term* dterms;  /* PQ_PARAM_POTENTIAL: dH/dtheta terms             */
    int nterms;
} pq_param_desc;

pq_status pq_survival_grad(pq_state* state, const pq_prop_desc* desc, int nsteps,
                           int ckpt_every, const pq_param_desc* params, int nparams,
                           double* grad_out, double* P_out, void* stream);

/* Observables of the state's current coefficients without any device
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that must not let a library call cudaMalloc / cudaFree, e.g. code
 * running under a framework allocator that owns the whole device-memory
 * budget, or step loops that must not pay the device-wide synchronisation an
 * allocation or free implies.
 *   out[0], out[1]  C = <Psi(0)|psi> (re, im), as in pq_observables_get;
 *   out[2]          ||psi||^2;
 *   out[3]          number of active points with |a| < theta (as a double).
 * `out` is a host array of 4 doubles; the call synchronises `stream`.
 * Scratch: a fixed 1 MiB file-scope device array (32768 blocks x 4 partial
 * sums), held by every GPU that loads the library until exit.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress)
 * with the device current; make that first call before any stream capture.
 * The array is shared by all calls and keeps the last call's contents: calls
 * that overlap on the GPU (other streams, other host threads) race on it.
 * DVR and projected-Weylet states only: a pvB state (Sec. 2.2) needs the
 * bra factors B^dagger f and the norm a^dagger S_AA a, which take full-grid
 * transforms, and is refused with PQ_ENOTSUP.
 * Errors: PQ_EINVAL for a null state or output, theta < 0, or more than
 * 268,435,456 active points (the scratch's limit); PQ_ENOTSUP for a pvB
 * state; PQ_ECAPACITY if the state's active set outgrew its capacity. */
pq_status pq_observe_noalloc(const pq_state* state, double theta, double* out, void* stream);

/* Device memory through the caller's allocator (no counterpart in the paper):
 * every device buffer the library takes (state buffers, the Krylov space,
 * temporaries of a propagation) is then obtained as alloc(bytes, stream, ctx)
 * and returned as free(ptr, stream, ctx), `stream` being the cudaStream_t the
 * buffer is used on (0 for long-lived buffers).  This lets a framework such as
 * PyTorch keep all device memory in its caching allocator.  alloc = free =
 * NULL restores cudaMalloc.  Host memory (one small pinned counter block per
 * state) and the fixed scratch of pq_observe_noalloc are not affected.
 * PQ_EINVAL while any state exists (a state must free with the allocator it
 * allocated with) or when only one of the two functions is given.  Not to be
 * called concurrently with other library calls. */
typedef void* (*pq_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*pq_free_fn)(void* ptr, void* stream, void* ctx);
pq_status pq_set_allocator(pq_alloc_fn alloc, pq_free_fn free_fn, void* ctx);

/* Arithmetic peak of the current device, measured (no counterpart in the
 * paper; the H.psi kernels are compared with it, next to the HBM bandwidth).
 * kind: PQ_PEAK_FP32 (scalar fused multiply-add), PQ_PEAK_FP32X2 (packed
 * two-lane FP32 FMA, sm_100 and later), PQ_PEAK_FP64.  The device runs
 * dependent FMA chains (8 per thread, `iters` FMAs each, 2048 threads per SM)
 * once untimed and once timed with CUDA events on the legacy default stream;
 * *ms_out receives the timed run's milliseconds and *flop_out its floating-
 * point operations (2 per FMA and lane).  Synchronises the device; allocates
 * a small device buffer.  Errors: PQ_EINVAL for an unknown kind, iters < 1 or
 * a null output; PQ_ECUDA. */
typedef enum pq_peak_kind { PQ_PEAK_FP32 = 0, PQ_PEAK_FP32X2 = 1, PQ_PEAK_FP64 = 2 } pq_peak_kind;
pq_status pq_measure_peak(int kind, int iters, double* ms_out, double* flop_out);

/* Number of kernels the library has launched since load (all states). */
int64_t pq_launch_count(void);

/* Message of the last failing call on this thread ("" if none). */
const char* pq_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PRUNEDQ_H */
