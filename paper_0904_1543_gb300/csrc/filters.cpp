// Host-side derivation of the Daubechies-16 filters used by the kernels.
//
// The paper prints no coefficient, so they are derived from their defining
// properties in double-double arithmetic (~106 bits) and rounded once:
//  * h_j, j = -7..8 (Eq. refinement): spectral factor of
//    |m0(xi)|^2 = cos^16(xi/2) P(sin^2(xi/2)), P(y) = sum_{k<8} C(7+k,k) y^k,
//    least-asymmetric member (phase of the non-trivial factor closest to
//    linear over (0, pi)); mirror images tie, the one with energy centre
//    sum_j j h_j^2 >= 1/2 is kept; sum_j h_j = sqrt 2.
//  * g_j = (-1)^j h_{1-j} (printed after Eq. refinement).
//  * magic filter w_k, k = k0..k0+15 (Eq. magicfilter): exact point values of
//    polynomials of degree < 16 from their scaling-function projections.
//    With D p = int p(. + y) phi(y) dy = sum_r m_r p^(r), m_r = M_r / r!, the
//    condition sum_k w_k (Dp)(-k) = p(0) gives w_k = (D^-1 l_k)(0), l_k the
//    Lagrange basis on the nodes -k and D^-1 = sum_r b_r d^r with
//    (sum m_r t^r)(sum b_r t^r) = 1.  k0 = round(M_1 - 7.5).
//  * kinetic a_l = int phi phi''(x - l) dx, |l| <= 14 (Eqs. kiner, fprod):
//    null vector of a_l = 4 sum_{i,j} h_i h_j a_{2l+j-i}, normalised by
//    sum_l l^2 a_l = 2.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <vector>

#include "wvl_internal.h"

namespace wvl {
namespace {

// ----------------------------------------------------------- double-double
struct dd {
    double hi, lo;
    dd() : hi(0), lo(0) {}
    dd(double h) : hi(h), lo(0) {}
    dd(double h, double l) : hi(h), lo(l) {}
};

inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return dd(s, e);
}
inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    return dd(s, b - (s - a));
}
inline dd two_prod(double a, double b) {
    double p = a * b;
    return dd(p, std::fma(a, b, -p));
}
inline dd operator+(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return dd(-a.hi, -a.lo); }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
inline dd operator/(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = a - b * dd(q1);
    double q2 = r.hi / b.hi;
    r = r - b * dd(q2);
    double q3 = r.hi / b.hi;
    return quick_two_sum(q1, q2) + dd(q3);
}
inline dd dsqrt(dd a) {
    if (a.hi <= 0) return dd(0);
    double x = std::sqrt(a.hi);
    dd r = a - two_prod(x, x);
    return quick_two_sum(x, r.hi / (2.0 * x)) ;
}
inline double dabs(dd a) { return std::fabs(a.hi); }

struct cdd {
    dd re, im;
    cdd() {}
    cdd(dd r, dd i) : re(r), im(i) {}
};
inline cdd operator+(cdd a, cdd b) { return cdd(a.re + b.re, a.im + b.im); }
inline cdd operator-(cdd a, cdd b) { return cdd(a.re - b.re, a.im - b.im); }
inline cdd operator*(cdd a, cdd b) {
    return cdd(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
inline cdd operator/(cdd a, cdd b) {
    dd d = b.re * b.re + b.im * b.im;
    return cdd((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
inline double cabs2d(cdd a) { return (a.re * a.re + a.im * a.im).hi; }
inline cdd csqrt(cdd a) {
    dd r = dsqrt(a.re * a.re + a.im * a.im);
    dd re = dsqrt((r + a.re) * dd(0.5));
    dd im = dsqrt((r - a.re) * dd(0.5));
    if (a.im.hi < 0) im = -im;
    return cdd(re, im);
}

double binom(int n, int k) {
    double r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// ----------------------------------------------------------- roots of P
constexpr int M = 8;       // vanishing moments
constexpr int NT = 16;     // taps of h
constexpr int JLO = -7;
constexpr int KH = 14;     // kinetic half width

std::vector<cdd> roots_of_P() {
    // monic coefficients of P(y) = sum_k C(7+k,k) y^k, degree 7
    const int deg = M - 1;
    std::vector<dd> c(deg + 1);
    double lead = binom(2 * M - 2, deg);
    for (int k = 0; k <= deg; ++k) c[k] = dd(binom(M - 1 + k, k)) / dd(lead);
    auto P = [&](cdd y) {
        cdd p(dd(1), dd(0));
        for (int k = deg - 1; k >= 0; --k) p = p * y + cdd(c[k], dd(0));
        return p;
    };
    // Durand-Kerner (Weierstrass) iteration from the usual start points
    std::vector<cdd> z(deg);
    std::complex<double> s0(0.4, 0.9), s = 1.0;
    for (int k = 0; k < deg; ++k) {
        z[k] = cdd(dd(s.real()), dd(s.imag()));
        s *= s0;
    }
    for (int it = 0; it < 400; ++it) {
        double move = 0;
        for (int k = 0; k < deg; ++k) {
            cdd den(dd(1), dd(0));
            for (int j = 0; j < deg; ++j)
                if (j != k) den = den * (z[k] - z[j]);
            cdd step = P(z[k]) / den;
            z[k] = z[k] - step;
            move = std::max(move, cabs2d(step));
        }
        if (move < 1e-64 && it > 20) break;
    }
    return z;
}

struct Cand {
    unsigned choice;
    std::vector<dd> h;     // j = -7..8
    std::vector<double> q; // ascending, real
    double crit;
};

double phase_nonlinearity(const std::vector<double>& q) {
    const int K = 4096;
    std::vector<double> xi(K - 1), th(K - 1);
    double prev = 0, acc = 0;
    for (int k = 1; k < K; ++k) {
        double x = M_PI * k / K;
        std::complex<double> zz = std::polar(1.0, -x), v = 0;
        for (int i = (int)q.size() - 1; i >= 0; --i) v = v * zz + q[i];
        double a = std::atan2(v.imag(), v.real());
        if (k == 1) {
            acc = a;
        } else {
            double d = a - prev;
            double dm = std::fmod(d + M_PI, 2 * M_PI);
            if (dm < 0) dm += 2 * M_PI;
            dm -= M_PI;
            if (dm == -M_PI && d > 0) dm = M_PI;
            acc += dm;
        }
        prev = a;
        xi[k - 1] = x;
        th[k - 1] = acc;
    }
    // least-squares line th ~ alpha xi + beta
    double n = K - 1, sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int i = 0; i < K - 1; ++i) {
        sx += xi[i]; sy += th[i]; sxx += xi[i] * xi[i]; sxy += xi[i] * th[i];
    }
    double alpha = (n * sxy - sx * sy) / (n * sxx - sx * sx);
    double beta = (sy - alpha * sx) / n;
    double m = 0;
    for (int i = 0; i < K - 1; ++i) m = std::max(m, std::fabs(th[i] - alpha * xi[i] - beta));
    return m;
}

Cand make_candidate(unsigned choice, const std::vector<cdd>& reals,
                    const std::vector<cdd>& cplx) {
    std::vector<cdd> zs;
    int bit = 0;
    auto zpair = [](cdd y, int outside) {
        cdd w(dd(1) - dd(2) * y.re, -(dd(2) * y.im));
        cdd d = csqrt(w * w - cdd(dd(1), dd(0)));
        cdd z1 = w + d, z2 = w - d;
        bool z1in = cabs2d(z1) < cabs2d(z2);
        cdd in = z1in ? z1 : z2, out = z1in ? z2 : z1;
        return outside ? out : in;
    };
    for (const cdd& y : reals) zs.push_back(zpair(y, (choice >> bit++) & 1));
    for (const cdd& y : cplx) {
        cdd z = zpair(y, (choice >> bit++) & 1);
        zs.push_back(z);
        zs.push_back(cdd(z.re, -z.im));
    }
    std::vector<cdd> q(1, cdd(dd(1), dd(0)));
    for (const cdd& zk : zs) {
        std::vector<cdd> nq(q.size() + 1, cdd(dd(0), dd(0)));
        for (size_t i = 0; i < q.size(); ++i) {
            nq[i + 1] = nq[i + 1] + q[i];
            nq[i] = nq[i] - q[i] * zk;
        }
        q.swap(nq);
    }
    Cand c;
    c.choice = choice;
    std::vector<dd> qr(q.size());
    for (size_t i = 0; i < q.size(); ++i) qr[i] = q[i].re;
    std::vector<dd> hz(qr.size() + M, dd(0));
    for (size_t i = 0; i < qr.size(); ++i)
        for (int k = 0; k <= M; ++k) hz[i + k] = hz[i + k] + qr[i] * dd(binom(M, k));
    dd sum(0);
    for (auto& v : hz) sum = sum + v;
    dd scale = dsqrt(dd(2)) / sum;
    for (auto& v : hz) c.h.push_back(v * scale);
    for (auto& v : qr) c.q.push_back(v.hi);
    c.crit = phase_nonlinearity(c.q);
    return c;
}

// solves the homogeneous system A x = 0 (rank n-1) for its null vector by
// Gaussian elimination with complete pivoting
std::vector<dd> null_vector(std::vector<std::vector<dd>> A) {
    const int n = (int)A.size();
    std::vector<int> col(n);
    for (int i = 0; i < n; ++i) col[i] = i;
    for (int k = 0; k < n - 1; ++k) {
        int pr = k, pc = k;
        double best = -1;
        for (int r = k; r < n; ++r)
            for (int cc = k; cc < n; ++cc)
                if (dabs(A[r][cc]) > best) { best = dabs(A[r][cc]); pr = r; pc = cc; }
        std::swap(A[k], A[pr]);
        if (pc != k) {
            for (int r = 0; r < n; ++r) std::swap(A[r][k], A[r][pc]);
            std::swap(col[k], col[pc]);
        }
        for (int r = k + 1; r < n; ++r) {
            dd f = A[r][k] / A[k][k];
            for (int cc = k; cc < n; ++cc) A[r][cc] = A[r][cc] - f * A[k][cc];
        }
    }
    // the last pivot vanishes; the last (permuted) unknown is free
    std::vector<dd> y(n, dd(0));
    y[n - 1] = dd(1);
    for (int r = n - 2; r >= 0; --r) {
        dd s(0);
        for (int cc = r + 1; cc < n; ++cc) s = s + A[r][cc] * y[cc];
        y[r] = -s / A[r][r];
    }
    std::vector<dd> x(n);
    for (int i = 0; i < n; ++i) x[col[i]] = y[i];
    return x;
}

FilterSet derive() {
    FilterSet F{};
    std::vector<cdd> all = roots_of_P();
    std::vector<cdd> reals, cplx;
    for (const cdd& y : all) {
        double im = y.im.hi, mag = std::max(1.0, std::fabs(y.re.hi));
        if (std::fabs(im) < 1e-20 * mag) reals.push_back(cdd(y.re, dd(0)));
        else if (im > 0) cplx.push_back(y);
    }
    std::sort(reals.begin(), reals.end(), [](const cdd& a, const cdd& b) { return a.re.hi < b.re.hi; });
    std::sort(cplx.begin(), cplx.end(), [](const cdd& a, const cdd& b) {
        return a.re.hi < b.re.hi || (a.re.hi == b.re.hi && a.im.hi < b.im.hi);
    });
    const int ngrp = (int)(reals.size() + cplx.size());
    std::vector<Cand> cands;
    for (unsigned ch = 0; ch < (1u << ngrp); ++ch) cands.push_back(make_candidate(ch, reals, cplx));
    size_t ib = 0;
    for (size_t i = 1; i < cands.size(); ++i)
        if (cands[i].crit < cands[ib].crit) ib = i;
    unsigned mirror = (~cands[ib].choice) & ((1u << ngrp) - 1);
    const Cand* pick = &cands[ib];
    double centre = 0;
    for (int t = 0; t < NT; ++t) centre += (JLO + t) * pick->h[t].hi * pick->h[t].hi;
    if (centre < 0.5) {
        for (const Cand& c : cands)
            if (c.choice == mirror) pick = &c;
    }
    std::vector<dd> h = pick->h;
    for (int t = 0; t < NT; ++t) {
        F.h[t] = h[t].hi + h[t].lo;
        int j = JLO + t;
        double v = h[(1 - j) - JLO].hi + h[(1 - j) - JLO].lo;
        F.g[t] = (j % 2 == 0) ? v : -v;
    }

    // moments M_p, p < 16
    std::vector<dd> Mo(NT);
    Mo[0] = dd(1);
    dd r2 = dsqrt(dd(2));
    for (int p = 1; p < NT; ++p) {
        dd acc(0);
        for (int t = 0; t < NT; ++t) {
            int j = JLO + t;
            dd inner(0);
            for (int q = 0; q < p; ++q) {
                double jp = std::pow((double)j, p - q);   // exact: |j|^15 < 2^53
                inner = inner + dd(binom(p, q)) * dd(jp) * Mo[q];
            }
            acc = acc + h[t] * inner;
        }
        dd two_p = dd(std::ldexp(1.0, p));
        Mo[p] = acc / (two_p * r2) / (dd(1) - dd(1) / two_p);
    }
    const int k0 = (int)std::lround(Mo[1].hi - 7.5);
    F.k0 = k0;

    // w_k = sum_r b_r r! [x^r] l_k(x)
    std::vector<dd> m(NT), b(NT);
    double fact = 1;
    for (int r = 0; r < NT; ++r) {
        if (r > 0) fact *= r;
        m[r] = Mo[r] / dd(fact);
    }
    b[0] = dd(1);
    for (int r = 1; r < NT; ++r) {
        dd s(0);
        for (int q = 1; q <= r; ++q) s = s + m[q] * b[r - q];
        b[r] = -s;
    }
    for (int t = 0; t < NT; ++t) {
        const int k = k0 + t;
        std::vector<double> num(1, 1.0);   // prod_{k' != k} (x + k'), exact integers
        double den = 1;
        for (int u = 0; u < NT; ++u) {
            if (u == t) continue;
            const int kp = k0 + u;
            std::vector<double> nn(num.size() + 1, 0.0);
            for (size_t i = 0; i < num.size(); ++i) {
                nn[i + 1] += num[i];
                nn[i] += num[i] * kp;
            }
            num.swap(nn);
            den *= (double)(kp - k);
        }
        dd acc(0);
        double rf = 1;
        for (int r = 0; r < NT; ++r) {
            if (r > 0) rf *= r;
            acc = acc + b[r] * dd(rf) * dd(num[r]);
        }
        dd wk = acc / dd(den);
        F.w[t] = wk.hi + wk.lo;
    }

    // kinetic: (I - 4R) a = 0, R_{l,m} = r(m - 2l), r(k) = sum_i h_i h_{i+k}
    std::vector<dd> rc(2 * NT - 1, dd(0));
    for (int k = -(NT - 1); k <= NT - 1; ++k)
        for (int i = 0; i < NT; ++i)
            if (i + k >= 0 && i + k < NT) rc[k + NT - 1] = rc[k + NT - 1] + h[i] * h[i + k];
    const int NK = 2 * KH + 1;
    std::vector<std::vector<dd>> A(NK, std::vector<dd>(NK, dd(0)));
    for (int l = -KH; l <= KH; ++l)
        for (int mm = -KH; mm <= KH; ++mm) {
            int k = mm - 2 * l;
            dd v = (k >= -(NT - 1) && k <= NT - 1) ? dd(-4) * rc[k + NT - 1] : dd(0);
            if (mm == l) v = v + dd(1);
            A[l + KH][mm + KH] = v;
        }
    std::vector<dd> a = null_vector(A);
    dd norm(0);
    for (int l = -KH; l <= KH; ++l) norm = norm + dd((double)(l * l)) * a[l + KH];
    for (int i = 0; i < NK; ++i) {
        dd v = a[i] * dd(2) / norm;
        F.a[i] = v.hi + v.lo;
    }
    return F;
}

}  // namespace

const FilterSet& filters() {
    static FilterSet F;
    static std::once_flag once;
    std::call_once(once, [] { F = derive(); });
    return F;
}

}  // namespace wvl
