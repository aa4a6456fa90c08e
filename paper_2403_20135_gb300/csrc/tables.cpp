// Host-side FP64 precompute: Gauss grid, normalised associated Legendre
// table, recurrence coefficients, Radau-right collocation data, FFT plans and
// twiddles.  Runs once in sdc_create; everything here is uploaded to the
// device and never recomputed on the hot path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sdc_internal.h"

namespace sdc {

namespace {

// P_n(x) and P_n'(x) by the Bonnet recurrence (n >= 1).
void legendre_value_and_slope(int n, double x, double &p, double &dp) {
    double pm1 = 1.0, pn = x;
    for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * x * pn - (k - 1.0) * pm1) / k;
        pm1 = pn;
        pn = pk;
    }
    p = pn;
    // (1 - x^2) P_n'(x) = n (P_{n-1}(x) - x P_n(x))
    dp = n * (pm1 - x * pn) / ((1.0 - x) * (1.0 + x));
}

}  // namespace

// Gauss-Legendre rule on [-1, 1], nodes ordered north to south (mu
// descending).  Newton's method runs in the colatitude theta = acos(mu) so
// that the polar nodes and weights keep full relative precision; the weight
// is 2 / ((1 - mu^2) P_J'(mu)^2) with 1 - mu^2 = sin^2(theta).
void gauss_legendre(int J, std::vector<double> &mu, std::vector<double> &w) {
    mu.assign(J, 0.0);
    w.assign(J, 0.0);
    const int half = (J + 1) / 2;
    for (int i = 0; i < half; ++i) {
        double th = M_PI * (i + 0.75) / (J + 0.5);
        for (int it = 0; it < 40; ++it) {
            const double x = std::cos(th);
            double p, dp;
            legendre_value_and_slope(J, x, p, dp);
            // d/dtheta P_J(cos theta) = -sin(theta) P_J'(x)
            const double delta = p / (-std::sin(th) * dp);
            th -= delta;
            if (std::fabs(delta) <= 1e-17) break;
        }
        const double x = std::cos(th);
        const double s = std::sin(th);
        double p, dp;
        legendre_value_and_slope(J, x, p, dp);
        // keep the (1 - x^2) P' product intact: n (P_{n-1} - x P_n) / sin(theta)
        const double slope_times_s = dp * ((1.0 - x) * (1.0 + x)) / s;
        const double wi = 2.0 / (slope_times_s * slope_times_s);
        mu[i] = x;
        w[i] = wi;
        mu[J - 1 - i] = -x;
        w[J - 1 - i] = wi;
    }
    if (J % 2 == 1) mu[J / 2] = 0.0;
}

// Radau IIA (right) nodes on [0, 1]: tau_M = 1 and the M - 1 roots of
// P_M(x) - P_{M-1}(x) in (-1, 1), mapped by tau = (x + 1) / 2.  The roots are
// bracketed on a fine grid and refined by bisection.  Q[m][j] integrates the
// Lagrange basis l_j over [0, tau_m] with an M-point Gauss rule (exact for
// polynomials of degree <= 2M - 1).
void radau_right(int M, std::vector<double> &tau, std::vector<double> &Q) {
    tau.assign(M, 0.0);
    Q.assign(M * M, 0.0);
    auto f = [M](double x) {
        double p0 = 1.0, p1 = x;
        if (M == 1) return p1 - p0;
        for (int k = 2; k <= M; ++k) {
            double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        return p1 - p0;
    };
    int found = 0;
    const int ngrid = 20000;
    double xa = -1.0, fa = f(xa);
    for (int g = 1; g <= ngrid && found < M - 1; ++g) {
        double xb = -1.0 + 2.0 * g / ngrid * (1.0 - 1e-9);
        double fb = f(xb);
        if (fa == 0.0 || (fa < 0) != (fb < 0)) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                double fm = f(mid);
                if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
            }
            tau[found++] = 0.5 * (0.5 * (lo + hi) + 1.0);
        }
        xa = xb;
        fa = fb;
    }
    tau[M - 1] = 1.0;
    std::vector<double> gx, gw;
    gauss_legendre(M, gx, gw);
    for (int m = 0; m < M; ++m) {
        for (int j = 0; j < M; ++j) {
            double acc = 0.0;
            for (int q = 0; q < M; ++q) {
                double s = 0.5 * tau[m] * (gx[q] + 1.0);
                double l = 1.0;
                for (int k = 0; k < M; ++k)
                    if (k != j) l *= (s - tau[k]) / (tau[j] - tau[k]);
                acc += gw[q] * l;
            }
            Q[m * M + j] = 0.5 * tau[m] * acc;
        }
    }
}

// Determinant of the square submatrix of the M x M row-major A kept by the
// index mask `keep` (Gaussian elimination with partial pivoting; 1 for none).
static double masked_det(const std::vector<double> &A, int M, unsigned keep) {
    int idx[16], n = 0;
    for (int i = 0; i < M; ++i)
        if (keep & (1u << i)) idx[n++] = i;
    double a[16][16];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) a[r][c] = A[idx[r] * M + idx[c]];
    double det = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (std::fabs(a[r][k]) > std::fabs(a[piv][k])) piv = r;
        if (a[piv][k] == 0.0) return 0.0;
        if (piv != k) {
            for (int c = 0; c < n; ++c) std::swap(a[k][c], a[piv][c]);
            det = -det;
        }
        det *= a[k][k];
        for (int r = k + 1; r < n; ++r) {
            const double f = a[r][k] / a[k][k];
            for (int c = k; c < n; ++c) a[r][c] -= f * a[k][c];
        }
    }
    return det;
}

// MIN-SR-S diagonal: the positive, increasing d_1 < ... < d_M for which the
// stiff-limit sweep matrix I - D^{-1} Q is nilpotent, i.e. every eigenvalue
// of D^{-1} Q is 1, i.e. det(x Q - D) = det(Q) (x - 1)^M.  Comparing the
// coefficients of x^{M-k} gives, for k = 1..M,
//   sum over index sets S of size k of (prod_{i in S} d_i) det(Q with S's rows and columns removed)
//     = C(M, k) det(Q),
// solved by damped Newton in y = log d (keeps d positive) from d = 2 tau / M,
// each equation scaled by C(M, k) |det Q|.  Returns false if the iteration
// does not reach such a root (d increasing, ||(I - D^{-1}Q)^M|| < 1e-9).
bool min_sr_s_diagonal(int M, const std::vector<double> &tau, const std::vector<double> &Q, std::vector<double> &d) {
    if (M < 1 || M > 8) return false;
    d.assign(M, 0.0);
    const unsigned full = (1u << M) - 1u;
    std::vector<double> minor(1u << M);                   // det of Q without the rows/columns in S
    for (unsigned S = 0; S <= full; ++S) minor[S] = masked_det(Q, M, full & ~S);
    const double detQ = minor[0];
    double binom[9] = {1, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 1; k <= M; ++k) binom[k] = binom[k - 1] * (M - k + 1) / k;
    std::vector<double> y(M), F(M), J(M * M), step(M);
    for (int i = 0; i < M; ++i) y[i] = std::log(2.0 * tau[i] / M);
    auto residual = [&](const std::vector<double> &yy, std::vector<double> &FF, std::vector<double> *JJ) {
        std::fill(FF.begin(), FF.end(), 0.0);
        if (JJ) std::fill(JJ->begin(), JJ->end(), 0.0);
        for (unsigned S = 1; S <= full; ++S) {
            int k = 0;
            double sumy = 0.0;
            for (int i = 0; i < M; ++i)
                if (S & (1u << i)) { ++k; sumy += yy[i]; }
            const double term = std::exp(sumy) * minor[S];
            FF[k - 1] += term;
            if (JJ)
                for (int i = 0; i < M; ++i)
                    if (S & (1u << i)) (*JJ)[(k - 1) * M + i] += term;
        }
        double nrm = 0.0;
        for (int k = 1; k <= M; ++k) {
            const double sc = binom[k] * std::fabs(detQ);
            FF[k - 1] = (FF[k - 1] - binom[k] * detQ) / sc;
            if (JJ)
                for (int i = 0; i < M; ++i) (*JJ)[(k - 1) * M + i] /= sc;
            nrm += FF[k - 1] * FF[k - 1];
        }
        return std::sqrt(nrm);
    };
    std::vector<double> yt(M), Ft(M);
    for (int it = 0; it < 100; ++it) {
        const double f0 = residual(y, F, &J);
        if (!std::isfinite(f0)) return false;
        // solve J step = F (partial pivoting on a copy)
        std::vector<double> A = J, b = F;
        for (int k = 0; k < M; ++k) {
            int piv = k;
            for (int r = k + 1; r < M; ++r)
                if (std::fabs(A[r * M + k]) > std::fabs(A[piv * M + k])) piv = r;
            if (A[piv * M + k] == 0.0) return false;
            if (piv != k) {
                for (int c = 0; c < M; ++c) std::swap(A[k * M + c], A[piv * M + c]);
                std::swap(b[k], b[piv]);
            }
            for (int r = k + 1; r < M; ++r) {
                const double f = A[r * M + k] / A[k * M + k];
                for (int c = k; c < M; ++c) A[r * M + c] -= f * A[k * M + c];
                b[r] -= f * b[k];
            }
        }
        for (int k = M - 1; k >= 0; --k) {
            double acc = b[k];
            for (int c = k + 1; c < M; ++c) acc -= A[k * M + c] * step[c];
            step[k] = acc / A[k * M + k];
        }
        double lam = 1.0, f1 = f0;
        for (; lam > 1e-8; lam *= 0.5) {
            for (int i = 0; i < M; ++i) yt[i] = y[i] - lam * step[i];
            f1 = residual(yt, Ft, nullptr);
            if (std::isfinite(f1) && f1 < (1.0 - 1e-4 * lam) * f0) break;
        }
        if (lam <= 1e-8) break;                          // no descent left: converged or stuck
        double move = 0.0;
        for (int i = 0; i < M; ++i) {
            move = std::max(move, std::fabs(lam * step[i]));
            y[i] = yt[i];
        }
        if (move < 1e-14) break;
    }
    for (int i = 0; i < M; ++i) d[i] = std::exp(y[i]);
    for (int i = 1; i < M; ++i)
        if (!(d[i] > d[i - 1])) return false;
    // nilpotency check: (I - D^{-1} Q)^M
    std::vector<double> K(M * M), P(M * M, 0.0), T(M * M);
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < M; ++c) K[r * M + c] = (r == c ? 1.0 : 0.0) - Q[r * M + c] / d[r];
    P = K;
    for (int p = 1; p < M; ++p) {
        for (int r = 0; r < M; ++r)
            for (int c = 0; c < M; ++c) {
                double acc = 0.0;
                for (int k = 0; k < M; ++k) acc += P[r * M + k] * K[k * M + c];
                T[r * M + c] = acc;
            }
        P = T;
    }
    double worst = 0.0;
    for (double v : P) worst = std::max(worst, std::fabs(v));
    return worst < 1e-9;
}

// Implicit weights of the LU trick for serial SDC: Q^T = L U with L unit
// lower triangular (Doolittle, no pivoting), q^Delta = U^T (lower triangular).
bool lu_implicit_weights(int M, const std::vector<double> &Q, std::vector<double> &qd) {
    std::vector<double> A(M * M), U(M * M, 0.0), L(M * M, 0.0);
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < M; ++c) A[r * M + c] = Q[c * M + r];   // Q^T
    for (int i = 0; i < M; ++i) {
        for (int k = i; k < M; ++k) {
            double s = A[i * M + k];
            for (int j = 0; j < i; ++j) s -= L[i * M + j] * U[j * M + k];
            U[i * M + k] = s;
        }
        if (U[i * M + i] == 0.0) return false;
        L[i * M + i] = 1.0;
        for (int k = i + 1; k < M; ++k) {
            double s = A[k * M + i];
            for (int j = 0; j < i; ++j) s -= L[k * M + j] * U[j * M + i];
            L[k * M + i] = s / U[i * M + i];
        }
    }
    qd.assign(M * M, 0.0);
    for (int r = 0; r < M; ++r)
        for (int c = 0; c <= r; ++c) qd[r * M + c] = U[c * M + r];
    return true;
}

// Normalised associated Legendre functions (unit L2 norm on [-1, 1], no
// Condon-Shortley phase) at the northern Gauss latitudes, degrees m..T+1.
// Pbar_0^0 = 1/sqrt(2), Pbar_m^m = sqrt((2m+1)/(2m)) sqrt(1-mu^2) Pbar_{m-1}^{m-1},
// Pbar_n^m = (mu Pbar_{n-1}^m - eps_{n-1}^m Pbar_{n-2}^m) / eps_n^m.
void legendre_table(int T, int J2, int J2p, const std::vector<double> &mu, std::vector<double> &table) {
    const int next = (T + 1) * (T + 4) / 2;
    table.assign(static_cast<size_t>(next) * J2p, 0.0);
    std::vector<double> eps;
    epsilon_table(T, eps);
    for (int j = 0; j < J2; ++j) {
        const double x = mu[j];
        const double s = std::sqrt((1.0 - x) * (1.0 + x));
        double pmm = 1.0 / std::sqrt(2.0);
        for (int m = 0; m <= T; ++m) {
            if (m > 0) pmm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
            const int base = ext_offset(T, m);
            double p2 = 0.0, p1 = pmm;
            table[static_cast<size_t>(base) * J2p + j] = pmm;
            for (int n = m + 1; n <= T + 1; ++n) {
                const double e_n = eps[base + n - m];
                const double e_n1 = eps[base + n - 1 - m];
                const double p = (x * p1 - e_n1 * p2) / e_n;
                table[static_cast<size_t>(base + n - m) * J2p + j] = p;
                p2 = p1;
                p1 = p;
            }
        }
    }
}

// Tables of the on-the-fly Legendre recurrence of the FP32 synthesis, every
// value split into an FP32 pair (hi = the FP32 rounding, lo = the FP32
// rounding of the remainder):
//   ab[e] = (a_hi, a_lo, b_hi, b_lo) of Pbar_n = a_n mu Pbar_{n-1} - b_n Pbar_{n-2},
//           a_n = 1 / eps_n, b_n = eps_{n-1} / eps_n (row e of degree n >= m + 2),
//   seed[m][j] = (Pbar_m^m, Pbar_{m+1}^m) at latitude j (from the FP64 table),
//   mu2[j] = mu_j (zero for the padding latitudes j >= J2).
void recurrence_tables(int T, int J2, int J2p, const std::vector<double> &mu, const std::vector<double> &table,
                       std::vector<float> &ab, std::vector<float> &seed, std::vector<float> &mu2) {
    const int next = (T + 1) * (T + 4) / 2;
    std::vector<double> eps;
    epsilon_table(T, eps);
    auto split = [](double x, float *o) {
        const float hi = static_cast<float>(x);
        o[0] = hi;
        o[1] = static_cast<float>(x - static_cast<double>(hi));
    };
    ab.assign(4 * static_cast<size_t>(next), 0.0f);
    for (int m = 0; m <= T; ++m) {
        const int base = ext_offset(T, m);
        for (int n = m + 2; n <= T + 1; ++n) {
            const int e = base + n - m;
            split(1.0 / eps[e], &ab[4 * static_cast<size_t>(e)]);
            split(eps[e - 1] / eps[e], &ab[4 * static_cast<size_t>(e) + 2]);
        }
    }
    seed.assign(4 * static_cast<size_t>(T + 1) * J2p, 0.0f);
    for (int m = 0; m <= T; ++m) {
        const int base = ext_offset(T, m);
        for (int j = 0; j < J2; ++j) {
            float *o = &seed[4 * (static_cast<size_t>(m) * J2p + j)];
            split(table[static_cast<size_t>(base) * J2p + j], o);
            split(table[static_cast<size_t>(base + 1) * J2p + j], o + 2);
        }
    }
    mu2.assign(2 * static_cast<size_t>(J2p), 0.0f);
    for (int j = 0; j < J2; ++j) split(mu[j], &mu2[2 * static_cast<size_t>(j)]);
}

void epsilon_table(int T, std::vector<double> &eps) {
    const int next = (T + 1) * (T + 4) / 2;
    eps.assign(next, 0.0);
    for (int m = 0; m <= T; ++m)
        for (int n = m; n <= T + 1; ++n) {
            const double nn = n, mm = m;
            eps[ext_offset(T, m) + n - m] = n == 0 ? 0.0 : std::sqrt((nn * nn - mm * mm) / (4.0 * nn * nn - 1.0));
        }
}

// Factors that map (zeta, div) on degrees m..T to the coefficients of the
// wind components U = u cos(lat), V = v cos(lat) on degrees n' = m..T+1:
//   U_n' = i c0 div_n' - c1 zeta_{n'-1} - c2 zeta_{n'+1}
//   V_n' = i c0 zeta_n' + c1 div_{n'-1} + c2 div_{n'+1}
// with s_n = -a^2 / (n(n+1)) (the inverse Laplacian, 0 at n = 0 and outside
// m..T), c0 = (m/a) s_n', c1 = -(n'-1) eps_n' s_{n'-1} / a,
// c2 = (n'+2) eps_{n'+1} s_{n'+1} / a.  This is U = (1/a) sum_n [i m chi_n Pbar_n
// - psi_n H_n] (and V alike) after H_n = -n eps_{n+1} Pbar_{n+1} + (n+1) eps_n Pbar_{n-1}.
void synthesis_factors(int T, double a, std::vector<double> &syn) {
    const int next = (T + 1) * (T + 4) / 2;
    syn.assign(3 * static_cast<size_t>(next), 0.0);
    std::vector<double> eps;
    epsilon_table(T, eps);
    for (int m = 0; m <= T; ++m) {
        const int base = ext_offset(T, m);
        auto s = [&](int n) { return (n < m || n > T || n == 0) ? 0.0 : -a * a / (double(n) * double(n + 1)); };
        for (int n = m; n <= T + 1; ++n) {
            const int e = base + n - m;
            syn[3 * e] = double(m) / a * s(n);
            syn[3 * e + 1] = (n - 1 >= m) ? -(n - 1.0) * eps[e] * s(n - 1) / a : 0.0;
            syn[3 * e + 2] = (n + 1 <= T) ? (n + 2.0) * eps[e + 1] * s(n + 1) / a : 0.0;
        }
    }
}

void order_maps(int T, std::vector<int> &row_m, std::vector<int> &coef_m) {
    row_m.clear();
    coef_m.clear();
    for (int m = 0; m <= T; ++m) {
        for (int n = m; n <= T + 1; ++n) row_m.push_back(m);
        for (int n = m; n <= T; ++n) coef_m.push_back(m);
    }
}

namespace {

// Round to the nearest BF16 (ties to even) through the float bit pattern.
uint16_t to_bf16(double x) {
    const float f = static_cast<float>(x);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return static_cast<uint16_t>(u >> 16);   // inf / nan
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return static_cast<uint16_t>(u >> 16);
}

double from_bf16(uint16_t h) {
    const uint32_t u = static_cast<uint32_t>(h) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// x = sum of npieces BF16 values, each the rounded residual of the previous.
void split_pieces(double x, int npieces, uint16_t *out) {
    double r = x;
    for (int i = 0; i < npieces; ++i) {
        out[i] = to_bf16(r);
        r -= from_bf16(out[i]);
    }
}

}  // namespace

// Pre-split Legendre operands of the tensor-core contractions (see TcTables).
// Analysis tiles: group (m, p) rows in tiles of 128, K = latitudes padded to
// 16 (kj), chunks of kTcChunkKB k-blocks; synthesis tiles: latitudes in
// tiles of 128, K = the group's rows padded to 16.
void build_tc_tables(int T, int J2, int J2p, const std::vector<double> &pbar, int npieces,
                     std::vector<uint16_t> &a3, std::vector<TcTile3> &tiles3, std::vector<uint16_t> &a1,
                     std::vector<TcTile1> &tiles1, int *kj_out) {
    const int kj = (J2 + 15) / 16 * 16;
    const int kjb = kj / 8;
    *kj_out = kj;
    tiles3.clear();
    tiles1.clear();
    long long n3 = 0, n1 = 0;
    for (int m = 0; m <= T; ++m)
        for (int p = 0; p < 2; ++p) {
            const int R = (T + 2 - m - p + 1) / 2;      // n' = m + p + 2q <= T + 1
            if (R <= 0) continue;
            for (int q0 = 0; q0 < R; q0 += 128) {
                TcTile3 t{m, p, q0, std::min(128, R - q0), 0, n3};
                t.nrb = (t.nrows + 7) / 8;
                tiles3.push_back(t);
                n3 += static_cast<long long>(t.nrb) * kjb * 64;
            }
            const int KR = (R + 15) / 16 * 16;
            for (int j0 = 0; j0 < J2; j0 += 128) {
                TcTile1 t{m, p, j0, std::min(128, J2 - j0), 0, R, KR, n1};
                t.njb = (t.nj + 7) / 8;
                tiles1.push_back(t);
                n1 += static_cast<long long>(t.njb) * (KR / 8) * 64;
            }
        }
    a3.assign(static_cast<size_t>(n3) * npieces, 0);
    a1.assign(static_cast<size_t>(n1) * npieces, 0);
    uint16_t pc[4];
    auto P = [&](int m, int n, int j) { return pbar[static_cast<size_t>(ext_offset(T, m) + n - m) * J2p + j]; };
    for (const TcTile3 &t : tiles3) {
        // chunk c: k blocks [8c, 8c + kbc); layout [rb][kb < kbc][8][8] per chunk
        long long off = t.aoff;
        for (int c0 = 0; c0 < kjb; c0 += kTcChunkKB) {
            const int kbc = std::min(kTcChunkKB, kjb - c0);
            for (int rb = 0; rb < t.nrb; ++rb)
                for (int kb = 0; kb < kbc; ++kb)
                    for (int r8 = 0; r8 < 8; ++r8)
                        for (int k8 = 0; k8 < 8; ++k8) {
                            const int q = t.q0 + rb * 8 + r8;
                            const int j = (c0 + kb) * 8 + k8;
                            double v = 0.0;
                            if (q < t.q0 + t.nrows && j < J2) v = P(t.m, t.m + t.p + 2 * q, j);
                            split_pieces(v, npieces, pc);
                            const long long e = off + ((rb * kbc + kb) * 8 + r8) * 8 + k8;
                            for (int i = 0; i < npieces; ++i) a3[static_cast<size_t>(i) * n3 + e] = pc[i];
                        }
            off += static_cast<long long>(t.nrb) * kbc * 64;
        }
    }
    for (const TcTile1 &t : tiles1) {
        const int krb = t.KR / 8;
        long long off = t.aoff;
        for (int c0 = 0; c0 < krb; c0 += kTcChunkKB) {
            const int kbc = std::min(kTcChunkKB, krb - c0);
            for (int jb = 0; jb < t.njb; ++jb)
                for (int kb = 0; kb < kbc; ++kb)
                    for (int r8 = 0; r8 < 8; ++r8)
                        for (int k8 = 0; k8 < 8; ++k8) {
                            const int j = t.j0 + jb * 8 + r8;
                            const int q = (c0 + kb) * 8 + k8;
                            double v = 0.0;
                            if (j < t.j0 + t.nj && q < t.R) v = P(t.m, t.m + t.p + 2 * q, j);
                            split_pieces(v, npieces, pc);
                            const long long e = off + ((jb * kbc + kb) * 8 + r8) * 8 + k8;
                            for (int i = 0; i < npieces; ++i) a1[static_cast<size_t>(i) * n1 + e] = pc[i];
                        }
            off += static_cast<long long>(t.njb) * kbc * 64;
        }
    }
}

bool fft_plan(int L, FftPlan &plan) {
    plan.L = L;
    plan.nstages = 0;
    int rest = L;
    while (rest % 8 == 0 && plan.nstages < kMaxStages) { plan.radix[plan.nstages++] = 8; rest /= 8; }
    if (rest % 4 == 0 && plan.nstages < kMaxStages) { plan.radix[plan.nstages++] = 4; rest /= 4; }
    if (rest % 2 == 0 && plan.nstages < kMaxStages) { plan.radix[plan.nstages++] = 2; rest /= 2; }
    while (rest % 3 == 0) {
        if (plan.nstages >= kMaxStages) return false;
        plan.radix[plan.nstages++] = 3;
        rest /= 3;
    }
    return rest == 1 && plan.nstages <= kMaxStages;
}

bool fft_plan16(int L, FftPlan &plan) {
    plan.L = L;
    plan.nstages = 0;
    int rest = L;
    while (rest % 16 == 0 && plan.nstages < kMaxStages) { plan.radix[plan.nstages++] = 16; rest /= 16; }
    for (int r : {8, 4, 2})
        if (rest % r == 0 && plan.nstages < kMaxStages) { plan.radix[plan.nstages++] = r; rest /= r; }
    while (rest % 3 == 0) {
        if (plan.nstages >= kMaxStages) return false;
        plan.radix[plan.nstages++] = 3;
        rest /= 3;
    }
    return rest == 1;
}

void pass_twiddles(const FftPlan &plan, const std::vector<double> &re, const std::vector<double> &im,
                   std::vector<double> &pre, std::vector<double> &pim) {
    pre.clear();
    pim.clear();
    int Ns = plan.radix[0];
    for (int p = 1; p < plan.nstages; ++p) {
        const int R = plan.radix[p];
        const int tws = plan.L / (Ns * R);
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < Ns; ++k) {
                pre.push_back(re[static_cast<size_t>(r) * k * tws]);
                pim.push_back(im[static_cast<size_t>(r) * k * tws]);
            }
        Ns *= R;
    }
}

// e^{-2 pi i k / L}: the angle is folded into [0, pi/4] with exact integer
// arithmetic before calling sin/cos.
void twiddles(int L, std::vector<double> &re, std::vector<double> &im) {
    re.assign(L, 0.0);
    im.assign(L, 0.0);
    const double unit = 2.0 * M_PI / (8.0 * L);   // angle of 1/(8L) of a turn
    for (int k = 0; k < L; ++k) {
        // angle = 2 pi k / L = unit * 8k; work with a = 8k in [0, 8L)
        long long a = 8LL * k;
        double sgn_s = 1.0;
        if (a > 4LL * L) { a = 8LL * L - a; sgn_s = -1.0; }         // theta -> 2pi - theta
        double sgn_c = 1.0;
        if (a > 2LL * L) { a = 4LL * L - a; sgn_c = -1.0; }         // theta -> pi - theta
        double c, s;
        if (a > L) {                                                 // theta -> pi/2 - theta
            const double t = unit * static_cast<double>(2LL * L - a);
            c = std::sin(t);
            s = std::cos(t);
        } else {
            const double t = unit * static_cast<double>(a);
            c = std::cos(t);
            s = std::sin(t);
        }
        re[k] = sgn_c * c;
        im[k] = -sgn_s * s;    // forward kernel e^{-i theta}
    }
}

}  // namespace sdc
