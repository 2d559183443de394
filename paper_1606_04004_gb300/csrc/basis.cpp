// Host-side (FP64) construction of the 1D primitive bases and packet factors.
// Sec. 2.1: the wavefunction is expanded in direct products of DVR functions
// chi_j (points x_j, weights w_j); Sec. 2.2 (Eq. pvN_def): a function f
// projects onto chi_j with the coefficient sqrt(w_j) f(x_j).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "pq_internal.h"

namespace pq {

// Cyclic Jacobi eigendecomposition of a symmetric n x n matrix A (row-major,
// destroyed).  On return evals ascending and evecs column j = eigenvector j.
// Returns the number of sweeps used (< 0 if it did not converge).
int jacobi_eigh(int n, std::vector<double>& A, std::vector<double>& evals,
                std::vector<double>& evecs) {
    evecs.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) evecs[(size_t)i * n + i] = 1.0;
    int sweep = 0;
    for (; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i) {
            diag += A[(size_t)i * n + i] * A[(size_t)i * n + i];
            for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        }
        if (off <= 1e-32 * (diag + 1e-300)) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                // rotation angle that zeroes A_pq: tan(2 phi) = 2 apq / (aqq - app)
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {   // V <- V J
                    double vkp = evecs[(size_t)k * n + p], vkq = evecs[(size_t)k * n + q];
                    evecs[(size_t)k * n + p] = c * vkp - s * vkq;
                    evecs[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    // sort ascending
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(),
              [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
    evals.resize(n);
    std::vector<double> V2((size_t)n * n);
    for (int j = 0; j < n; ++j) {
        evals[j] = A[(size_t)order[j] * n + order[j]];
        for (int k = 0; k < n; ++k) V2[(size_t)k * n + j] = evecs[(size_t)k * n + order[j]];
    }
    evecs.swap(V2);
    return sweep < 100 ? sweep : -1;
}

// Sine DVR on [xmin, xmax]: particle-in-a-box functions diagonalised in x.
static void sine_dvr(int n, double xmin, double xmax, double mass, std::vector<double>& x,
                     std::vector<double>& w, std::vector<double>& T) {
    const double L = xmax - xmin;
    x.resize(n);
    w.assign(n, L / (n + 1));
    for (int j = 0; j < n; ++j) x[j] = xmin + (j + 1) * L / (n + 1);
    T.assign((size_t)n * n, 0.0);
    const double pref = 2.0 / (n + 1);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double acc = 0.0;
            for (int k = 1; k <= n; ++k) {
                double ek = (k * M_PI / L) * (k * M_PI / L) / (2.0 * mass);
                acc += sin((a + 1) * k * M_PI / (n + 1)) * ek * sin((b + 1) * k * M_PI / (n + 1));
            }
            T[(size_t)a * n + b] = pref * acc;
        }
}

// Fourier grid (FGH) DVR on the periodic box [xmin, xmax): x_j = xmin + j L/n,
// w = L/n, T_ij = (1/n) sum_l (k_l^2 / 2m) cos(k_l (x_i - x_j)), k_l = 2 pi l / L,
// l = -(n-1)/2 .. n/2 (integer division; for even n the last is the Nyquist mode).
static void fgh_dvr(int n, double xmin, double xmax, double mass, std::vector<double>& x,
                    std::vector<double>& w, std::vector<double>& T) {
    const double L = xmax - xmin;
    x.resize(n);
    w.assign(n, L / n);
    for (int j = 0; j < n; ++j) x[j] = xmin + j * L / n;
    T.assign((size_t)n * n, 0.0);
    const int lo = -((n - 1) / 2), hi = n / 2;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double acc = 0.0;
            for (int l = lo; l <= hi; ++l) {
                const double k = 2.0 * M_PI * l / L;
                acc += k * k / (2.0 * mass) * cos(2.0 * M_PI * (double)l * (a - b) / n);
            }
            T[(size_t)a * n + b] = acc / n;
        }
}

// Normalised HO functions phi_0..phi_{n} at x (three-term recurrence in
// xi = sqrt(m omega) x): phi_{k+1} = sqrt(2/(k+1)) xi phi_k - sqrt(k/(k+1)) phi_{k-1}.
static void ho_functions(int n, double mass, double omega, double x, double* phi) {
    const double xi = sqrt(mass * omega) * x;
    phi[0] = pow(mass * omega / M_PI, 0.25) * exp(-0.5 * xi * xi);
    if (n >= 1) phi[1] = sqrt(2.0) * xi * phi[0];
    for (int k = 1; k < n; ++k)
        phi[k + 1] = sqrt(2.0 / (k + 1)) * xi * phi[k] - sqrt((double)k / (k + 1)) * phi[k - 1];
}

// HO (Gauss-Hermite) DVR: the DVR points are the eigenvalues of the position
// matrix in the first n oscillator functions, i.e. the zeros of phi_n (found
// by Jacobi, then polished by Newton on phi_n).  The transformation is
// U_ki = sqrt(w_i) phi_k(x_i) with w_i = 1 / sum_k phi_k(x_i)^2 (the DVR
// weight that turns grid values into coefficients); evaluating it from the
// recurrence keeps full relative accuracy in the small edge components.
// Kinetic energy exact in the oscillator basis, then transformed: T = U^T K U.
static int ho_dvr(int n, double mass, double omega, std::vector<double>& x,
                  std::vector<double>& w, std::vector<double>& T) {
    std::vector<double> X((size_t)n * n, 0.0), Uj, ev;
    for (int k = 0; k + 1 < n; ++k)
        X[(size_t)k * n + k + 1] = X[(size_t)(k + 1) * n + k] = sqrt((k + 1) / (2.0 * mass * omega));
    if (jacobi_eigh(n, X, ev, Uj) < 0) return -1;
    std::vector<double> phi(n + 2);
    const double s = sqrt(mass * omega);
    for (int i = 0; i < n; ++i) {
        double xi = ev[i];
        for (int it = 0; it < 4; ++it) {   // Newton on phi_n: phi_n' = s (sqrt(n/2) phi_{n-1} - sqrt((n+1)/2) phi_{n+1})
            ho_functions(n + 1, mass, omega, xi, phi.data());
            const double d = s * (sqrt(n / 2.0) * phi[n - 1] - sqrt((n + 1) / 2.0) * phi[n + 1]);
            if (d == 0.0) break;
            xi -= phi[n] / d;
        }
        ev[i] = xi;
    }
    std::vector<double> U((size_t)n * n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        ho_functions(n - 1, mass, omega, ev[i], phi.data());
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += phi[k] * phi[k];
        w[i] = 1.0 / acc;
        const double sw = sqrt(w[i]);
        for (int k = 0; k < n; ++k) U[(size_t)k * n + i] = sw * phi[k];
    }
    std::vector<double> K((size_t)n * n, 0.0);   // p^2 / (2 m) in the HO basis
    for (int k = 0; k < n; ++k) K[(size_t)k * n + k] = mass * omega * (k + 0.5) / (2.0 * mass);
    for (int k = 0; k + 2 < n; ++k) {
        double v = -0.5 * mass * omega * sqrt((k + 1.0) * (k + 2.0)) / (2.0 * mass);
        K[(size_t)k * n + k + 2] = K[(size_t)(k + 2) * n + k] = v;
    }
    T.assign((size_t)n * n, 0.0);
    std::vector<double> KU((size_t)n * n, 0.0);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += K[(size_t)a * n + k] * U[(size_t)k * n + b];
            KU[(size_t)a * n + b] = acc;
        }
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += U[(size_t)k * n + a] * KU[(size_t)k * n + b];
            T[(size_t)a * n + b] = acc;
        }
    for (int a = 0; a < n; ++a)   // symmetrise rounding
        for (int b = a + 1; b < n; ++b) {
            double m = 0.5 * (T[(size_t)a * n + b] + T[(size_t)b * n + a]);
            T[(size_t)a * n + b] = T[(size_t)b * n + a] = m;
        }
    x = ev;
    return 0;
}

// Projected Weylets (Sec. 2.4) on a sine or FGH DVR: momentum-symmetrised Gaussians
// (Eq. sG_def, Sec. 2.3) on the doubly dense lattice Dx Dp = pi (x_a cell-centred,
// p_b = (b + 1/2) Dp > 0, alpha = Dp / (2 Dx)), projected on the DVR
// (Phi_ji = sqrt(w_j) phi_i(x_j), i = a np + b) and orthogonalised
// symmetrically: W = Phi S^(-1/2), S = Phi^T Phi.  W (n x n, row-major) maps
// pW coefficients to DVR coefficients.
pq_status build_pw_mode(const pq_mode_desc& m, std::vector<double>& x, std::vector<double>& w,
                        std::vector<double>& T, std::vector<double>& W) {
    const int n = m.n, nx = m.nx_lattice, np_ = m.np_lattice;
    if (n < 2 || n > kMaxN) {
        set_error("projected Weylets: %d functions per mode outside 2..%d", n, kMaxN);
        return PQ_EINVAL;
    }
    if (nx < 1 || np_ < 1 || nx * np_ != n) {
        set_error("projected Weylets need nx_lattice * np_lattice = n (%d x %d != %d)", nx, np_, n);
        return PQ_EINVAL;
    }
    if (!(m.xmax > m.xmin) || !(m.mass > 0)) {
        set_error("projected Weylets need xmax > xmin and mass > 0");
        return PQ_EINVAL;
    }
    if (m.dvr == PQ_FGH_DVR) fgh_dvr(n, m.xmin, m.xmax, m.mass, x, w, T);
    else sine_dvr(n, m.xmin, m.xmax, m.mass, x, w, T);
    const double L = m.xmax - m.xmin, dx = L / nx, dp = M_PI / dx, alpha = dp / (2.0 * dx);
    const double shift = sqrt(M_PI / (8.0 * alpha)), amp = pow(8.0 * alpha / M_PI, 0.25);
    std::vector<double> Phi((size_t)n * n);
    for (int a = 0; a < nx; ++a) {
        const double xa = m.xmin + (a + 0.5) * dx;
        for (int b = 0; b < np_; ++b) {
            const double pb = (b + 0.5) * dp;
            for (int j = 0; j < n; ++j) {
                const double d = x[j] - xa;
                Phi[(size_t)j * n + a * np_ + b] =
                    sqrt(w[j]) * (amp * exp(-alpha * d * d) * sin(pb * (d - shift)));
            }
        }
    }
    std::vector<double> S((size_t)n * n, 0.0), U, lam;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc += Phi[(size_t)j * n + p] * Phi[(size_t)j * n + q];
            S[(size_t)p * n + q] = acc;
        }
    if (jacobi_eigh(n, S, lam, U) < 0) {
        set_error("projected Weylets: eigensolver of the overlap did not converge");
        return PQ_ENUMERIC;
    }
    for (int i = 0; i < n; ++i)
        if (!(lam[i] > 1e-12 * lam[n - 1])) {
            set_error("projected Weylets: overlap matrix is singular (lambda_min %.3e)", lam[0]);
            return PQ_ENUMERIC;
        }
    std::vector<double> Sm((size_t)n * n, 0.0);   // S^(-1/2) = U diag(lam^-1/2) U^T
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i)
                acc += U[(size_t)p * n + i] * U[(size_t)q * n + i] / sqrt(lam[i]);
            Sm[(size_t)p * n + q] = acc;
        }
    W.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j)
        for (int q = 0; q < n; ++q) {
            double acc = 0.0;
            for (int p = 0; p < n; ++p) acc += Phi[(size_t)j * n + p] * Sm[(size_t)p * n + q];
            W[(size_t)j * n + q] = acc;
        }
    return PQ_OK;
}

// Complex Gauss-Jordan inverse with partial pivoting (A: n x n interleaved
// re/im, row-major; replaced by its inverse).  Returns false if singular.
static bool complex_inverse(int n, std::vector<double>& A) {
    std::vector<double> I((size_t)n * n * 2, 0.0);
    for (int i = 0; i < n; ++i) I[((size_t)i * n + i) * 2] = 1.0;
    auto at = [n](std::vector<double>& M, int r, int c) { return &M[((size_t)r * n + c) * 2]; };
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = 0.0;
        for (int r = c; r < n; ++r) {
            const double* v = at(A, r, c);
            const double m = v[0] * v[0] + v[1] * v[1];
            if (m > best) {
                best = m;
                piv = r;
            }
        }
        if (!(best > 0.0)) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(at(A, c, k)[0], at(A, piv, k)[0]);
                std::swap(at(A, c, k)[1], at(A, piv, k)[1]);
                std::swap(at(I, c, k)[0], at(I, piv, k)[0]);
                std::swap(at(I, c, k)[1], at(I, piv, k)[1]);
            }
        const double pr = at(A, c, c)[0], pi = at(A, c, c)[1], d = pr * pr + pi * pi;
        const double ir = pr / d, ii = -pi / d;   // 1 / pivot
        for (int k = 0; k < n; ++k) {
            double* a = at(A, c, k);
            double* b = at(I, c, k);
            const double ar = a[0] * ir - a[1] * ii, ai = a[0] * ii + a[1] * ir;
            const double br = b[0] * ir - b[1] * ii, bi = b[0] * ii + b[1] * ir;
            a[0] = ar; a[1] = ai; b[0] = br; b[1] = bi;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double fr = at(A, r, c)[0], fi = at(A, r, c)[1];
            if (fr == 0.0 && fi == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                double* a = at(A, r, k);
                const double* ac = at(A, c, k);
                a[0] -= fr * ac[0] - fi * ac[1];
                a[1] -= fr * ac[1] + fi * ac[0];
                double* b = at(I, r, k);
                const double* bc = at(I, c, k);
                b[0] -= fr * bc[0] - fi * bc[1];
                b[1] -= fr * bc[1] + fi * bc[0];
            }
        }
    }
    A.swap(I);
    return true;
}

// Biorthogonal projected von Neumann basis (Sec. 2.2) on a sine DVR: von
// Neumann Gaussians (on a sine or FGH DVR) on the lattice Dx Dp = 2 pi (x_a cell-centred, momenta
// p_b = -p_max + (b + 1/2) Dp, p_max = np Dp / 2, alpha = Dp / (2 Dx)),
// projected (Eq. pvN_def): G_jm = sqrt(w_j) g_m(x_j); B = G^{-dagger}
// (Eq. pvb_def: B^dagger G = 1); S = B^dagger B.  Complex n x n, interleaved.
pq_status build_pvb_mode(const pq_mode_desc& m, std::vector<double>& x, std::vector<double>& w,
                         std::vector<double>& T, std::vector<double>& G, std::vector<double>& B,
                         std::vector<double>& S) {
    const int n = m.n, nx = m.nx_lattice, np_ = m.np_lattice;
    if (n < 2 || n > kMaxN) {
        set_error("pvB: %d functions per mode outside 2..%d", n, kMaxN);
        return PQ_EINVAL;
    }
    if (nx < 1 || np_ < 1 || nx * np_ != n) {
        set_error("pvB needs nx_lattice * np_lattice = n (%d x %d != %d)", nx, np_, n);
        return PQ_EINVAL;
    }
    if (!(m.xmax > m.xmin) || !(m.mass > 0)) {
        set_error("pvB needs xmax > xmin and mass > 0");
        return PQ_EINVAL;
    }
    if (m.dvr == PQ_FGH_DVR) fgh_dvr(n, m.xmin, m.xmax, m.mass, x, w, T);
    else sine_dvr(n, m.xmin, m.xmax, m.mass, x, w, T);
    const double L = m.xmax - m.xmin, dx = L / nx, dp = 2.0 * M_PI / dx, alpha = dp / (2.0 * dx);
    const double pmax = np_ * dp / 2.0, amp = pow(2.0 * alpha / M_PI, 0.25);
    G.assign((size_t)n * n * 2, 0.0);
    for (int a = 0; a < nx; ++a) {
        const double xa = m.xmin + (a + 0.5) * dx;
        for (int b = 0; b < np_; ++b) {
            const double pb = -pmax + (b + 0.5) * dp;
            for (int j = 0; j < n; ++j) {
                const double d = x[j] - xa;
                const double mag = sqrt(w[j]) * (amp * exp(-alpha * d * d));
                G[((size_t)j * n + a * np_ + b) * 2] = mag * cos(pb * d);
                G[((size_t)j * n + a * np_ + b) * 2 + 1] = mag * sin(pb * d);
            }
        }
    }
    std::vector<double> Gi = G;
    if (!complex_inverse(n, Gi)) {
        set_error("pvB: the projected von Neumann matrix G is singular");
        return PQ_ENUMERIC;
    }
    B.assign((size_t)n * n * 2, 0.0);   // B = (G^-1)^dagger
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            B[((size_t)i * n + j) * 2] = Gi[((size_t)j * n + i) * 2];
            B[((size_t)i * n + j) * 2 + 1] = -Gi[((size_t)j * n + i) * 2 + 1];
        }
    S.assign((size_t)n * n * 2, 0.0);   // S = B^dagger B
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < n; ++k) {
                const double ar = B[((size_t)k * n + p) * 2], ai = -B[((size_t)k * n + p) * 2 + 1];
                const double br = B[((size_t)k * n + q) * 2], bi = B[((size_t)k * n + q) * 2 + 1];
                sr += ar * br - ai * bi;
                si += ar * bi + ai * br;
            }
            S[((size_t)p * n + q) * 2] = sr;
            S[((size_t)p * n + q) * 2 + 1] = si;
        }
    return PQ_OK;
}

pq_status build_dvr_mode(const pq_mode_desc& m, std::vector<double>& x, std::vector<double>& w,
                         std::vector<double>& T) {
    if (m.n < 2 || m.n > kMaxN) {
        set_error("mode size %d outside 2..%d", m.n, kMaxN);
        return PQ_EINVAL;
    }
    if (!(m.mass > 0)) {
        set_error("mode mass must be positive");
        return PQ_EINVAL;
    }
    if (m.kind == PQ_SINE_DVR) {
        if (!(m.xmax > m.xmin)) {
            set_error("sine DVR needs xmax > xmin");
            return PQ_EINVAL;
        }
        sine_dvr(m.n, m.xmin, m.xmax, m.mass, x, w, T);
        return PQ_OK;
    }
    if (m.kind == PQ_FGH_DVR) {
        if (!(m.xmax > m.xmin)) {
            set_error("FGH DVR needs xmax > xmin");
            return PQ_EINVAL;
        }
        fgh_dvr(m.n, m.xmin, m.xmax, m.mass, x, w, T);
        return PQ_OK;
    }
    if (m.kind == PQ_HO_DVR) {
        if (!(m.omega > 0)) {
            set_error("HO DVR needs omega > 0");
            return PQ_EINVAL;
        }
        if (ho_dvr(m.n, m.mass, m.omega, x, w, T) != 0) {
            set_error("HO DVR eigensolver did not converge");
            return PQ_ENUMERIC;
        }
        return PQ_OK;
    }
    set_error("unknown basis kind %d", m.kind);
    return PQ_EINVAL;
}

// f_k(i) = sqrt(w_i) (2 pi s^2)^(-1/4) exp(-(x_i - q0)^2/(4 s^2) + i p0 (x_i - q0)),
// normalised per mode so that the full-lattice product has unit norm.
void packet_factors(const Basis& b, const double* q0, const double* p0, const double* width,
                    std::vector<double>& out, int lead_virtual) {
    const int Dint = b.D_user + lead_virtual;
    out.assign((size_t)Dint * kMaxN * 2, 0.0);
    if (lead_virtual) out[0] = 1.0;   // virtual size-1 mode: factor 1
    for (int k = 0; k < b.D_user; ++k) {
        const int n = b.modes[k].n;
        double* f = &out[(size_t)(k + lead_virtual) * kMaxN * 2];
        const double s2 = width[k] * width[k];
        const double amp = pow(2.0 * M_PI * s2, -0.25);
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) {
            double dx = b.x[k][i] - q0[k];
            double mag = sqrt(b.w[k][i]) * amp * exp(-dx * dx / (4.0 * s2));
            double ph = p0[k] * dx;
            f[2 * i] = mag * cos(ph);
            f[2 * i + 1] = mag * sin(ph);
            nrm += f[2 * i] * f[2 * i] + f[2 * i + 1] * f[2 * i + 1];
        }
        nrm = sqrt(nrm);
        for (int i = 0; i < 2 * n; ++i) f[i] /= nrm;
        if (!b.Gc[k].empty()) {   // pvB coefficients: G^dagger f (Eq. psi_exp_pvb)
            std::vector<double> g(2 * n, 0.0);
            const std::vector<double>& M = b.Gc[k];
            for (int q = 0; q < n; ++q)
                for (int j = 0; j < n; ++j) {
                    const double mr = M[((size_t)j * n + q) * 2], mi = -M[((size_t)j * n + q) * 2 + 1];
                    g[2 * q] += mr * f[2 * j] - mi * f[2 * j + 1];
                    g[2 * q + 1] += mr * f[2 * j + 1] + mi * f[2 * j];
                }
            for (int i = 0; i < 2 * n; ++i) f[i] = g[i];
        }
        if (!b.W[k].empty()) {   // pW coefficients: W^T f
            std::vector<double> g(2 * n, 0.0);
            for (int q = 0; q < n; ++q)
                for (int j = 0; j < n; ++j) {
                    g[2 * q] += b.W[k][(size_t)j * n + q] * f[2 * j];
                    g[2 * q + 1] += b.W[k][(size_t)j * n + q] * f[2 * j + 1];
                }
            for (int i = 0; i < 2 * n; ++i) f[i] = g[i];
        }
    }
}

}  // namespace pq
