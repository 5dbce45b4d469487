// Symmetric eigen-decomposition on the host for the POD Gram matrices:
// Householder reduction to tridiagonal form followed by the implicit-shift
// QL iteration (Wilkinson; the classical EISPACK method), O(n^3) with a
// small constant.  Host-only, FP64.
#pragma once

#include <math.h>

#include <algorithm>
#include <vector>

namespace ptrom {

// A: n x n symmetric, row-major.  On return w holds the eigenvalues in
// descending order and V (n x n, row-major) the eigenvectors as columns.
// Returns false if the QL iteration did not converge.
inline bool symeig(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &V) {
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
    std::vector<double> d(n, 0.0), e(n, 0.0);
    // --- Householder tridiagonalisation; row i is reduced against columns < i
    for (int i = n - 1; i > 0; --i) {
        const int l = i - 1;
        double h = 0.0;
        if (l > 0) {
            double scale = 0.0;
            for (int k = 0; k <= l; ++k) scale += fabs(a(i, k));
            if (scale == 0.0) {
                e[i] = a(i, l);
            } else {
                for (int k = 0; k <= l; ++k) {
                    a(i, k) /= scale;
                    h += a(i, k) * a(i, k);
                }
                double f = a(i, l);
                double g = f >= 0.0 ? -sqrt(h) : sqrt(h);
                e[i] = scale * g;
                h -= f * g;
                a(i, l) = f - g;
                f = 0.0;
                for (int j = 0; j <= l; ++j) {
                    a(j, i) = a(i, j) / h;
                    double gg = 0.0;
                    for (int k = 0; k <= j; ++k) gg += a(j, k) * a(i, k);
                    for (int k = j + 1; k <= l; ++k) gg += a(k, j) * a(i, k);
                    e[j] = gg / h;
                    f += e[j] * a(i, j);
                }
                const double hh = f / (h + h);
                for (int j = 0; j <= l; ++j) {
                    const double fj = a(i, j);
                    const double gj = e[j] - hh * fj;
                    e[j] = gj;
                    for (int k = 0; k <= j; ++k) a(j, k) -= fj * e[k] + gj * a(i, k);
                }
            }
        } else {
            e[i] = a(i, l);
        }
        d[i] = h;
    }
    d[0] = 0.0;
    e[0] = 0.0;
    // --- accumulate the orthogonal transformation into A
    for (int i = 0; i < n; ++i) {
        const int l = i - 1;
        if (d[i] != 0.0) {
            for (int j = 0; j <= l; ++j) {
                double g = 0.0;
                for (int k = 0; k <= l; ++k) g += a(i, k) * a(k, j);
                for (int k = 0; k <= l; ++k) a(k, j) -= g * a(k, i);
            }
        }
        d[i] = a(i, i);
        a(i, i) = 1.0;
        for (int j = 0; j <= l; ++j) a(j, i) = a(i, j) = 0.0;
    }
    // --- implicit-shift QL on the tridiagonal (d, e), vectors accumulated in A
    for (int i = 1; i < n; ++i) e[i - 1] = e[i];
    if (n > 0) e[n - 1] = 0.0;
    // off-diagonal entries below 1e-18 of the matrix scale are deflated too (a
    // Gram matrix of decaying snapshots has eigenvalues down to underflow)
    double anorm = 0.0;
    for (int i = 0; i < n; ++i) anorm = std::max(anorm, fabs(d[i]) + fabs(e[i]));
    const double tiny = 1e-18 * anorm;
    for (int l = 0; l < n; ++l) {
        int iter = 0, m;
        do {
            for (m = l; m < n - 1; ++m) {
                const double dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) <= 1e-16 * dd || fabs(e[m]) <= tiny) break;
            }
            if (m != l) {
                if (iter++ == 200) return false;
                double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                double r = hypot(g, 1.0);
                g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? fabs(r) : -fabs(r)));
                double s = 1.0, c = 1.0, p = 0.0;
                int i;
                bool deflated = false;
                for (i = m - 1; i >= l; --i) {
                    double f = s * e[i];
                    const double b = c * e[i];
                    r = hypot(f, g);
                    e[i + 1] = r;
                    if (r == 0.0) {
                        d[i + 1] -= p;
                        e[m] = 0.0;
                        deflated = true;
                        break;
                    }
                    s = f / r;
                    c = g / r;
                    g = d[i + 1] - p;
                    r = (d[i] - g) * s + 2.0 * c * b;
                    p = s * r;
                    d[i + 1] = g + p;
                    g = c * r - b;
                    for (int k = 0; k < n; ++k) {
                        f = a(k, i + 1);
                        a(k, i + 1) = s * a(k, i) + c * f;
                        a(k, i) = c * a(k, i) - s * f;
                    }
                }
                if (deflated) continue;
                d[l] -= p;
                e[l] = g;
                e[m] = 0.0;
            }
        } while (m != l);
    }
    // --- sort descending
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return d[x] > d[y]; });
    w.resize(n);
    V.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        w[j] = d[ord[j]];
        for (int k = 0; k < n; ++k) V[(size_t)k * n + j] = a(k, ord[j]);
    }
    return true;
}

}  // namespace ptrom
