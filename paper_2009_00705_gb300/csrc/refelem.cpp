// Reference-element construction for the spectral element method (Section 3.1).
//
// Nodal set (a reading; the paper names Fekete points without giving them):
// Warburton's warp & blend nodes with alpha = 0 on triangles (edge nodes are
// Gauss-Lobatto-Legendre points, so neighbouring elements share nodes), GLL
// points in the vertical.  Quadrature: collapsed Gauss rule with p+1 points per
// direction on the triangle, p+1 Gauss-Legendre points in the vertical.
// Lagrange bases are formed from the orthonormal collapsed-coordinate (Dubiner)
// modal basis through the inverse Vandermonde matrix.
#include "refelem.hpp"

#include <cmath>
#include <stdexcept>

namespace sem {

namespace {

// Recurrence coefficients of the orthonormal Jacobi family:
// x p_n = a_{n+1} p_{n+1} + b_n p_n + a_n p_{n-1}.
double rec_a(int n, double a, double b) {
    if (n == 1) return 2.0 / (2.0 + a + b) * std::sqrt((1.0 + a) * (1.0 + b) / (3.0 + a + b));
    const double s = 2.0 * n + a + b;
    return 2.0 / s * std::sqrt(n * (n + a) * (n + b) * (n + a + b) / ((s - 1.0) * (s + 1.0)));
}
double rec_b(int n, double a, double b) {
    if (n == 0) return (b - a) / (a + b + 2.0);
    const double s = 2.0 * n + a + b;
    return (b * b - a * a) / (s * (s + 2.0));
}

void invert(std::vector<double>& M, int n) {
    // Gauss-Jordan elimination with partial pivoting, in place.
    std::vector<double> A(M), I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) throw std::runtime_error("singular Vandermonde matrix");
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[c * n + k], A[piv * n + k]);
                std::swap(I[c * n + k], I[piv * n + k]);
            }
        const double d = 1.0 / A[c * n + c];
        for (int k = 0; k < n; ++k) { A[c * n + k] *= d; I[c * n + k] *= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
        }
    }
    M = I;
}

// Dubiner modes psi_ij(r,s) = sqrt(2) P~_i^(0,0)(a) P~_j^(2i+1,0)(b) (1-b)^i and
// their r/s derivatives, a = 2(1+r)/(1-s) - 1 (a = -1 at the vertex s = 1), b = s.
void dubiner(int p, double r, double s, double* psi, double* pr, double* ps) {
    const double oms = 1.0 - s;
    const double a = (std::fabs(oms) > 1e-14) ? 2.0 * (1.0 + r) / oms - 1.0 : -1.0;
    const double b = s;
    const double rt2 = std::sqrt(2.0);
    int m = 0;
    for (int i = 0; i <= p; ++i) {
        const double fa = jacobi(i, 0, 0, a), dfa = djacobi(i, 0, 0, a);
        const double pw_i = std::pow(oms, i);
        const double pw_im1 = (i >= 1) ? std::pow(oms, i - 1) : 0.0;
        for (int j = 0; j + i <= p; ++j, ++m) {
            const double gb = jacobi(j, 2 * i + 1, 0, b), dgb = djacobi(j, 2 * i + 1, 0, b);
            psi[m] = rt2 * fa * gb * pw_i;
            if (i == 0) {
                pr[m] = 0.0;
                ps[m] = rt2 * fa * dgb;
            } else {
                pr[m] = rt2 * 2.0 * dfa * gb * pw_im1;
                ps[m] = rt2 * (dfa * (1.0 + a) * gb * pw_im1 + fa * dgb * pw_i - i * fa * gb * pw_im1);
            }
        }
    }
}

}  // namespace

double jacobi(int n, double a, double b, double x) {
    const double mu0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0)
                       / std::tgamma(a + b + 2.0);
    double pm1 = 0.0, p0 = 1.0 / std::sqrt(mu0);
    for (int k = 0; k < n; ++k) {
        const double pn = ((x - rec_b(k, a, b)) * p0 - (k > 0 ? rec_a(k, a, b) * pm1 : 0.0)) / rec_a(k + 1, a, b);
        pm1 = p0;
        p0 = pn;
    }
    return p0;
}

double djacobi(int n, double a, double b, double x) {
    if (n == 0) return 0.0;
    return std::sqrt(n * (n + a + b + 1.0)) * jacobi(n - 1, a + 1.0, b + 1.0, x);
}

void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = std::acos(-1.0);
    for (int k = 0; k < n; ++k) {
        double r = -std::cos((2.0 * k + 1.0) * pi / (2.0 * n));
        if (k > 0) r = 0.5 * (r + x[k - 1]);
        for (int it = 0; it < 200; ++it) {
            double defl = 0.0;
            for (int j = 0; j < k; ++j) defl += 1.0 / (r - x[j]);
            const double f = jacobi(n, a, b, r), df = djacobi(n, a, b, r);
            const double del = -f / (df - defl * f);
            r += del;
            if (std::fabs(del) < 1e-17) break;
        }
        x[k] = r;
    }
    // sort ascending (roots come out ascending already; keep it robust)
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && x[j] < x[j - 1]; --j) std::swap(x[j], x[j - 1]);
    // Christoffel numbers of the orthonormal family
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) {
            const double v = jacobi(k, a, b, x[i]);
            s += v * v;
        }
        w[i] = 1.0 / s;
    }
}

std::vector<double> gll(int p) {
    std::vector<double> out(p + 1);
    out[0] = -1.0;
    out[p] = 1.0;
    if (p >= 2) {
        std::vector<double> x, w;
        gauss_jacobi(p - 1, 1.0, 1.0, x, w);   // interior GLL points: roots of L_p'
        for (int i = 0; i < p - 1; ++i) out[i + 1] = x[i];
    }
    return out;
}

void lagrange1d(const std::vector<double>& xn, const double* x, int npt,
                std::vector<double>& B, std::vector<double>& D) {
    const int n = (int)xn.size();
    std::vector<double> lam(n, 1.0);     // barycentric weights
    for (int k = 0; k < n; ++k)
        for (int m = 0; m < n; ++m)
            if (m != k) lam[k] /= (xn[k] - xn[m]);
    B.assign((size_t)npt * n, 0.0);
    D.assign((size_t)npt * n, 0.0);
    for (int q = 0; q < npt; ++q) {
        int hit = -1;
        for (int k = 0; k < n; ++k)
            if (x[q] == xn[k]) hit = k;
        if (hit >= 0) {
            for (int k = 0; k < n; ++k) {
                B[(size_t)q * n + k] = (k == hit) ? 1.0 : 0.0;
                if (k != hit) D[(size_t)q * n + k] = lam[k] / lam[hit] / (xn[hit] - xn[k]);
            }
            double s = 0.0;
            for (int m = 0; m < n; ++m)
                if (m != hit) s += 1.0 / (xn[hit] - xn[m]);
            D[(size_t)q * n + hit] = s;
            continue;
        }
        double den = 0.0;
        for (int k = 0; k < n; ++k) den += lam[k] / (x[q] - xn[k]);
        for (int k = 0; k < n; ++k) {
            const double l = lam[k] / (x[q] - xn[k]) / den;
            double s = 0.0;
            for (int m = 0; m < n; ++m)
                if (m != k) s += 1.0 / (x[q] - xn[m]);
            B[(size_t)q * n + k] = l;
            D[(size_t)q * n + k] = l * s;
        }
    }
}

std::vector<double> tri_nodes(int p) {
    const int NT = (p + 1) * (p + 2) / 2;
    std::vector<double> out(2 * NT);
    if (p == 0) { out[0] = out[1] = -1.0 / 3.0; return out; }
    const std::vector<double> g = gll(p);
    std::vector<double> eq(p + 1);
    for (int k = 0; k <= p; ++k) eq[k] = -1.0 + 2.0 * k / p;
    std::vector<double> disp(p + 1);
    for (int k = 0; k <= p; ++k) disp[k] = g[k] - eq[k];
    int n = 0;
    for (int j = 0; j <= p; ++j)
        for (int i = 0; i + j <= p; ++i, ++n) {
            const double mu[3] = {1.0 - double(i + j) / p, double(i) / p, double(j) / p};
            double nu[3] = {mu[0], mu[1], mu[2]};
            const int ea[3] = {0, 1, 2}, eb[3] = {1, 2, 0};
            for (int e = 0; e < 3; ++e) {
                const double tau = mu[eb[e]] - mu[ea[e]];
                double warp = 0.0;
                if (std::fabs(tau) < 1.0 - 1e-10) {
                    std::vector<double> Bq, Dq;
                    lagrange1d(eq, &tau, 1, Bq, Dq);
                    for (int k = 0; k <= p; ++k) warp += Bq[k] * disp[k];
                    warp /= (1.0 - tau * tau);
                }
                const double d = 4.0 * mu[ea[e]] * mu[eb[e]] * warp;
                nu[eb[e]] += 0.5 * d;
                nu[ea[e]] -= 0.5 * d;
            }
            out[2 * n] = -1.0 + 2.0 * nu[1];
            out[2 * n + 1] = -1.0 + 2.0 * nu[2];
        }
    return out;
}

void tri_lagrange(int p, const double* pts, int npt, std::vector<double>& B,
                  std::vector<double>& Dr, std::vector<double>& Ds) {
    const int NT = (p + 1) * (p + 2) / 2;
    const std::vector<double> nodes = tri_nodes(p);
    std::vector<double> V((size_t)NT * NT), tr(NT), ts(NT);
    for (int i = 0; i < NT; ++i) dubiner(p, nodes[2 * i], nodes[2 * i + 1], &V[(size_t)i * NT], tr.data(), ts.data());
    invert(V, NT);                         // V^{-1}[mode][node]
    B.assign((size_t)npt * NT, 0.0);
    Dr.assign((size_t)npt * NT, 0.0);
    Ds.assign((size_t)npt * NT, 0.0);
    std::vector<double> psi(NT), pr(NT), ps(NT);
    for (int q = 0; q < npt; ++q) {
        dubiner(p, pts[2 * q], pts[2 * q + 1], psi.data(), pr.data(), ps.data());
        for (int n = 0; n < NT; ++n) {
            double b = 0, dr = 0, ds = 0;
            for (int m = 0; m < NT; ++m) {
                const double v = V[(size_t)m * NT + n];
                b += psi[m] * v;
                dr += pr[m] * v;
                ds += ps[m] * v;
            }
            B[(size_t)q * NT + n] = b;
            Dr[(size_t)q * NT + n] = dr;
            Ds[(size_t)q * NT + n] = ds;
        }
    }
}

void RefLevel::build(int dim_, int p_, int pz_) {
    dim = dim_;
    p = p_;
    pz = (dim_ == 3 && pz_ > 0) ? pz_ : p_;
    NT = (p + 1) * (p + 2) / 2;
    tnodes = tri_nodes(p);
    const int n = p + 1;
    std::vector<double> ga, wa, gb, wb;
    gauss_jacobi(n, 0.0, 0.0, ga, wa);
    gauss_jacobi(n, 1.0, 0.0, gb, wb);
    QT = n * n;
    tq.resize(2 * QT);
    tw.resize(QT);
    for (int jb = 0; jb < n; ++jb)
        for (int ia = 0; ia < n; ++ia) {
            const int q = jb * n + ia;
            tq[2 * q] = 0.5 * (1.0 + ga[ia]) * (1.0 - gb[jb]) - 1.0;
            tq[2 * q + 1] = gb[jb];
            tw[q] = 0.5 * wa[ia] * wb[jb];
        }
    tri_lagrange(p, tq.data(), QT, Bt, Drt, Dst);
    face_nodes.clear();
    std::vector<int> tf[3];
    {
        int m = 0;
        for (int j = 0; j <= p; ++j)
            for (int i = 0; i + j <= p; ++i, ++m) {
                if (j == 0) tf[0].push_back(m);
                if (i + j == p) tf[1].push_back(m);
                if (i == 0) tf[2].push_back(m);
            }
    }
    if (dim == 2) {
        NZ = 1;
        QZ = 1;
        znodes = {0.0};
        zq = {0.0};
        zw = {1.0};
        Bz = {1.0};
        Dz = {0.0};
        Np = NT;
        Nq = QT;
        for (int f = 0; f < 3; ++f) face_nodes.push_back(tf[f]);
        return;
    }
    NZ = pz + 1;
    QZ = pz + 1;
    znodes = gll(pz);
    gauss_jacobi(QZ, 0.0, 0.0, zq, zw);
    lagrange1d(znodes, zq.data(), QZ, Bz, Dz);
    Np = NT * NZ;
    Nq = QT * QZ;
    for (int f = 0; f < 3; ++f) {
        std::vector<int> l;
        for (int k = 0; k < NZ; ++k)
            for (int m : tf[f]) l.push_back(k * NT + m);
        face_nodes.push_back(l);
    }
    std::vector<int> bot, top;
    for (int m = 0; m < NT; ++m) { bot.push_back(m); top.push_back(pz * NT + m); }
    face_nodes.push_back(bot);
    face_nodes.push_back(top);
}

void interp_factors(int dim, int pf, int pc, int pzf, int pzc, std::vector<double>& Bt, std::vector<double>& Bz) {
    const std::vector<double> fn = tri_nodes(pf);
    const int NTf = (pf + 1) * (pf + 2) / 2;
    std::vector<double> Dr, Ds;
    tri_lagrange(pc, fn.data(), NTf, Bt, Dr, Ds);
    if (dim == 2) {
        Bz.assign(1, 1.0);
        return;
    }
    const std::vector<double> zf = gll(pzf), zc = gll(pzc);
    std::vector<double> Dz;
    lagrange1d(zc, zf.data(), pzf + 1, Bz, Dz);
}

}  // namespace sem
