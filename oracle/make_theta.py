"""Write oracle/theta_tables.json: theta_m for m = 1..55 at tol = 2^-53 and 2^-24.

Definition (Al-Mohy & Higham 2011, Section 3; used by the paper's `step` and
`series`, Section 3.1): with T_m the degree-m Taylor polynomial of exp,

    h_{m+1}(x) = log(exp(-x) T_m(x)) = sum_{k >= m+1} c_k x^k,
    htilde_{m+1}(x) = sum_{k >= m+1} |c_k| x^k,

theta_m is the largest theta > 0 with htilde_{m+1}(theta) / theta <= tol.

The power series of exp(-x) T_m(x) is formed by direct multiplication of the two
series in 120-digit arithmetic, its logarithm by the standard series recurrence
(f = exp(g)  =>  k g_k = k f_k - sum_{j<k} j g_j f_{k-j} for f_0 = 1), and theta
by bisection on the monotone function htilde(theta)/theta - tol.
Run:  python oracle/make_theta.py   (needs mpmath; takes ~1 minute).
"""
import json
import os

import mpmath as mp

mp.mp.dps = 120
M_MAX = 55
EXTRA_TERMS = 300  # series truncated at k = m + EXTRA_TERMS (tail < 1e-60 at theta_m)


def log_series(m, kmax):
    e = [mp.mpf(-1) ** k / mp.factorial(k) for k in range(kmax + 1)]
    t = [1 / mp.factorial(j) for j in range(m + 1)]
    f = [mp.mpf(0)] * (kmax + 1)
    for i in range(kmax + 1):
        for j in range(min(m, kmax - i) + 1):
            f[i + j] += e[i] * t[j]
    g = [mp.mpf(0)] * (kmax + 1)
    for k in range(1, kmax + 1):
        acc = k * f[k]
        for j in range(1, k):
            acc -= j * g[j] * f[k - j]
        g[k] = acc / k
    return g


def theta(m, tol):
    kmax = m + EXTRA_TERMS
    c = log_series(m, kmax)
    absc = [abs(c[k]) for k in range(m + 1, kmax + 1)]

    def excess(th):
        return sum(a * th ** (k - 1) for a, k in zip(absc, range(m + 1, kmax + 1))) - tol

    lo, hi = mp.mpf(0), mp.mpf(1)
    while excess(hi) <= 0:
        lo, hi = hi, hi * 2
    for _ in range(260):
        mid = (lo + hi) / 2
        if excess(mid) <= 0:
            lo = mid
        else:
            hi = mid
    return lo


def main():
    out = {"definition": "largest theta with sum_{k>m} |c_k| theta^(k-1) <= tol, "
                         "c_k = Taylor coefficients of log(exp(-x) T_m(x))",
           "m_max": M_MAX}
    for name, tol in (("double", mp.mpf(2) ** -53), ("single", mp.mpf(2) ** -24)):
        out[name] = {"tol": float(tol),
                     "theta": [float(theta(m, tol)) for m in range(1, M_MAX + 1)]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "theta_tables.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
