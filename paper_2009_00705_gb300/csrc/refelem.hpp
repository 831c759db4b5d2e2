// Reference elements of the spectral element discretisation (Section 3.1):
// nodes, quadrature rules and Lagrange bases on the reference triangle
// T = {r, s >= -1, r + s <= 0} and the prism T x [-1, 1].
#pragma once
#include <vector>

namespace sem {

// L2-orthonormal Jacobi polynomial P~_n^(a,b)(x) on [-1,1] and its derivative.
double jacobi(int n, double a, double b, double x);
double djacobi(int n, double a, double b, double x);

// n-point Gauss-Jacobi rule for the weight (1-x)^a (1+x)^b (ascending nodes).
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
// p+1 Gauss-Lobatto-Legendre points (ascending).
std::vector<double> gll(int p);

// Warp & blend (alpha = 0) triangle nodes in lattice order (j outer, i inner), [NT][2].
std::vector<double> tri_nodes(int p);

// Order-p triangle Lagrange basis at npt points pts[npt][2]: B, Dr, Ds as [npt][NT].
void tri_lagrange(int p, const double* pts, int npt, std::vector<double>& B,
                  std::vector<double>& Dr, std::vector<double>& Ds);
// 1D Lagrange basis on nodes xn at points x: B, D as [npt][n].
void lagrange1d(const std::vector<double>& xn, const double* x, int npt,
                std::vector<double>& B, std::vector<double>& D);

// Everything the kernels of one order-p level need.
struct RefLevel {
    int dim = 3, p = 1, pz = 1;       // triangle order, vertical order (prisms; = p for triangles)
    int NT = 0, NZ = 1, QT = 0, QZ = 1, Np = 0, Nq = 0;
    std::vector<double> tnodes;      // [NT][2]
    std::vector<double> znodes;      // [NZ] GLL
    std::vector<double> tq, tw;      // tri quadrature points [QT][2], weights [QT]
    std::vector<double> zq, zw;      // vertical Gauss-Legendre points/weights [QZ]
    std::vector<double> Bt, Drt, Dst; // [QT][NT]
    std::vector<double> Bz, Dz;      // [QZ][NZ]
    std::vector<std::vector<int>> face_nodes;   // local node lists per face
    void build(int dim, int p, int pz = 0);   // pz = 0: the same order as p
};

// Element prolongation (the coarse basis at the fine nodes) in tensor factors: triangle
// part Bt [NT_f][NT_c] (orders pf -> pc) and vertical part Bz [NZ_f][NZ_c] (orders
// pzf -> pzc; [1] for triangles); I[(kf,nf)][(kc,nc)] = Bt[nf][nc] * Bz[kf][kc].
// Semi-coarsening lowers one of the two orders only.
void interp_factors(int dim, int pf, int pc, int pzf, int pzc, std::vector<double>& Bt, std::vector<double>& Bz);

}  // namespace sem
