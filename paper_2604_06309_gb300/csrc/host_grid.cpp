// Host FP64 construction of the theta grid (Sec. 3.2, Eq. theta) and of the
// quadrature weights nu (Sec. 3.4). O(L) work, done once per solver.
#include <cmath>
#include <vector>

#include "dmfe_internal.h"

// gamma = -W_{-1}(-1/t_max): root gamma > 1 of ln(gamma) - gamma + ln(t_max) = 0.
double host_gamma_from_tmax(double t_max) {
    const double lt = std::log(t_max);
    double lo = 1.0, hi = 2.0 * lt + 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (std::log(mid) - mid + lt > 0.0) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 3; ++it) x -= (std::log(x) - x + lt) / (1.0 / x - 1.0);
    return x;
}

// g_delta of Eq. (theta), taken odd so that theta(1) = 0 and theta(L) = 1.
static double g_delta(double x, double delta) {
    double v = std::cbrt(std::fabs(x) * x * x + delta * delta * delta) - delta;
    return x < 0 ? -v : v;
}

// theta(y) = [atan(e^{gamma y}) - atan(e^{-gamma})] / D, as a single atan of a quotient
// (no cancellation near theta = 0); 1 - theta(y) = theta(-y) by symmetry.
static double theta_of_y(double y, double gamma, double D) {
    double num = std::exp(-gamma) * std::expm1(gamma * (y + 1.0));
    double den = 1.0 + std::exp(gamma * (y - 1.0));
    return std::atan(num / den) / D;
}

void host_theta_grid(int L, double gamma, double alpha, double delta, std::vector<double>& theta,
                     std::vector<double>& omega) {
    theta.assign(L, 0.0);
    omega.assign(L, 0.0);
    const double D = std::atan(std::exp(gamma)) - std::atan(std::exp(-gamma));
    for (int k = 0; k < L; ++k) {
        double i = k + 1.0;
        double z = i;
        if (alpha != 0.0 && delta != 0.0) {
            double yi = (2.0 * i - 1.0 - L) / (L - 1.0);
            double phi = 0.5 * (L - 1.0) * (g_delta(yi, delta) / g_delta(1.0, delta) + 1.0) + 1.0;
            z = alpha * phi + (1.0 - alpha) * i;
        }
        double y = (2.0 * z - 1.0 - L) / (L - 1.0);
        theta[k] = theta_of_y(y, gamma, D);
        omega[k] = theta_of_y(-y, gamma, D);
    }
    theta[0] = 0.0; omega[0] = 1.0;
    theta[L - 1] = 1.0; omega[L - 1] = 0.0;
}

// nu_j = integral over [0,1] of the not-a-knot quintic spline through e_j (Sec. 3.4).
// With the collocation matrix A[r][c] = B_c(theta_r) and w_c = integral of B_c,
// nu solves A^T nu = w. A is a B-spline collocation matrix, hence totally positive,
// so banded Gaussian elimination without pivoting is stable.
int host_spline_weights(const std::vector<double>& x, std::vector<double>& nu) {
    const int k = 5;
    const int L = (int)x.size();
    if (L < k + 1) return DMFE_ERR_ARG;
    std::vector<double> t;
    for (int r = 0; r <= k; ++r) t.push_back(x[0]);
    for (int r = (k + 1) / 2; r < L - (k + 1) / 2; ++r) t.push_back(x[r]);
    for (int r = 0; r <= k; ++r) t.push_back(x[L - 1]);
    const int m = (int)t.size();  // L + 6 knots, L basis functions

    // Band of M = A^T: M[c][r] = B_c(x_r). Row r of A has its nonzeros in
    // c = mu_r - 5 .. mu_r with mu_r the knot span of x_r, so |c - r| <= 5.
    const int kl = 6, ku = 6, W = kl + ku + 1;
    std::vector<double> M((size_t)L * W, 0.0);
    auto at = [&](int row, int col) -> double& { return M[(size_t)row * W + (col - row + kl)]; };
    for (int r = 0; r < L; ++r) {
        const double xr = x[r];
        int mu = k;
        while (mu < m - k - 2 && t[mu + 1] <= xr) ++mu;  // t[mu] <= x < t[mu+1], last span at the end
        double N[k + 1], left[k + 1], right[k + 1];
        N[0] = 1.0;
        for (int d = 1; d <= k; ++d) {
            left[d] = xr - t[mu + 1 - d];
            right[d] = t[mu + d] - xr;
            double saved = 0.0;
            for (int q = 0; q < d; ++q) {
                double tmp = N[q] / (right[q + 1] + left[d - q]);
                N[q] = saved + right[q + 1] * tmp;
                saved = left[d - q] * tmp;
            }
            N[d] = saved;
        }
        for (int q = 0; q <= k; ++q) {
            int c = mu - k + q;
            if (c - r > ku || r - c > kl) return DMFE_ERR_ARG;
            at(c, r) = N[q];
        }
    }
    std::vector<double> rhs(L);
    for (int c = 0; c < L; ++c) rhs[c] = (t[c + k + 1] - t[c]) / (k + 1);
    // LU without pivoting inside the band, then the two triangular solves.
    for (int p = 0; p < L; ++p) {
        const double piv = at(p, p);
        if (!(std::fabs(piv) > 0.0)) return DMFE_ERR_ARG;
        for (int i = p + 1; i <= std::min(L - 1, p + kl); ++i) {
            double f = at(i, p) / piv;
            if (f == 0.0) continue;
            at(i, p) = f;
            for (int j = p + 1; j <= std::min(L - 1, p + ku); ++j) at(i, j) -= f * at(p, j);
        }
    }
    for (int i = 0; i < L; ++i)
        for (int j = std::max(0, i - kl); j < i; ++j) rhs[i] -= at(i, j) * rhs[j];
    for (int i = L - 1; i >= 0; --i) {
        double s = rhs[i];
        for (int j = i + 1; j <= std::min(L - 1, i + ku); ++j) s -= at(i, j) * rhs[j];
        rhs[i] = s / at(i, i);
    }
    nu = rhs;
    return DMFE_OK;
}
