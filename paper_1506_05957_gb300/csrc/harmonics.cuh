// Solid harmonics of the spherical-harmonic FMM (Sec. 2.5; the M_n^m and L_n^m
// expansions of the paper), with the Condon-Shortley phase:
//   R_n^m(x) = r^n P_n^m(cos t) e^{i m f} / (n+m)!      (regular)
//   I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m f} / r^{n+1}  (irregular)
//   X_n^{-m} = (-1)^m conj(X_n^m)
// With this scaling the translation theorems carry no extra factors:
//   1/|x - y|  = sum_{n,m} conj(R_n^m(y)) I_n^m(x),                |y| < |x|
//   R_n^m(a+b) = sum_{j,k} R_j^k(a) R_{n-j}^{m-k}(b)
//   I_n^m(t+a) = sum_{j,k} (-1)^j conj(R_j^k(a)) I_{n+j}^{m+k}(t),  |a| < |t|
//   (d/dx + i d/dy) R_n^m = R_{n-1}^{m+1},  d/dz R_n^m = R_{n-1}^m.
// Expansions: M_n^m = sum_j q_j conj(R_n^m(y_j - c)),  phi(x) = sum M_n^m I_n^m(x - c);
//             L_n^m = sum_j q_j conj(I_n^m(y_j - c)),  phi(x) = sum L_n^m R_n^m(x - c).
// Both tables are built column by column (fixed m, rising n) from Cartesian
// coordinates by the three-term Legendre recurrence: no trigonometry.
#pragma once
#include "common.cuh"

namespace fmmbem {

// out[cidx(n,m)] = R_n^m(x,y,z) for 0 <= m <= n <= p.
template <typename T>
FMM_HD void regular_table(T x, T y, T z, int p, cpx<T>* out) {
    const T r2 = x * x + y * y + z * z;
    cpx<T> diag = mk<T>(1, 0);
    const cpx<T> xy = mk(x, y);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) diag = (T(-0.5) / T(m)) * (xy * diag);
        out[cidx(m, m)] = diag;
        if (m + 1 > p) break;
        cpx<T> prev2 = diag, prev1 = z * diag;
        out[cidx(m + 1, m)] = prev1;
        for (int n = m + 2; n <= p; ++n) {
            const T inv = T(1) / T((n - m) * (n + m));
            cpx<T> cur = mk((T(2 * n - 1) * z * prev1.re - r2 * prev2.re) * inv,
                            (T(2 * n - 1) * z * prev1.im - r2 * prev2.im) * inv);
            out[cidx(n, m)] = cur;
            prev2 = prev1;
            prev1 = cur;
        }
    }
}

// out[cidx(n,m)] = I_n^m(x,y,z) for 0 <= m <= n <= p (x != 0).
template <typename T>
FMM_HD void irregular_table(T x, T y, T z, int p, cpx<T>* out) {
    const T r2 = x * x + y * y + z * z;
    const T ir2 = T(1) / r2;
    cpx<T> diag = mk<T>(sqrt(ir2), 0);
    const cpx<T> xy = mk(x, y);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) diag = (-T(2 * m - 1) * ir2) * (xy * diag);
        out[cidx(m, m)] = diag;
        if (m + 1 > p) break;
        cpx<T> prev2 = diag, prev1 = (T(2 * m + 1) * z * ir2) * diag;
        out[cidx(m + 1, m)] = prev1;
        for (int n = m + 2; n <= p; ++n) {
            const T a = T(2 * n - 1) * z, b = T((n + m - 1) * (n - m - 1));
            cpx<T> cur = mk((a * prev1.re - b * prev2.re) * ir2, (a * prev1.im - b * prev2.im) * ir2);
            out[cidx(n, m)] = cur;
            prev2 = prev1;
            prev1 = cur;
        }
    }
}

// Column m of the irregular table, degrees m..nmax, written to out[cidx(n,m)].
// Used when several threads build one table together (one column each).
template <typename T>
FMM_HD void irregular_column(T x, T y, T z, int m, int nmax, cpx<T>* out) {
    const T r2 = x * x + y * y + z * z;
    const T ir2 = T(1) / r2;
    cpx<T> diag = mk<T>(sqrt(ir2), 0);
    const cpx<T> xy = mk(x, y);
    for (int k = 1; k <= m; ++k) diag = (-T(2 * k - 1) * ir2) * (xy * diag);
    out[cidx(m, m)] = diag;
    if (m + 1 > nmax) return;
    cpx<T> prev2 = diag, prev1 = (T(2 * m + 1) * z * ir2) * diag;
    out[cidx(m + 1, m)] = prev1;
    for (int n = m + 2; n <= nmax; ++n) {
        const T a = T(2 * n - 1) * z, b = T((n + m - 1) * (n - m - 1));
        cpx<T> cur = mk((a * prev1.re - b * prev2.re) * ir2, (a * prev1.im - b * prev2.im) * ir2);
        out[cidx(n, m)] = cur;
        prev2 = prev1;
        prev1 = cur;
    }
}

// Coefficient X_n^m of a stored (m >= 0) table for any m in [-n, n].
template <typename T>
FMM_HD cpx<T> coef_any(const cpx<T>* tab, int n, int m) {
    if (m >= 0) return tab[cidx(n, m)];
    cpx<T> v = tab[cidx(n, -m)];
    return (m & 1) ? mk(-v.re, v.im) : mk(v.re, -v.im);
}

}  // namespace fmmbem
