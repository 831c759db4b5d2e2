// Host-side setup of a sem_handle: canonical numbering, Dirichlet sets,
// transfer bookkeeping, device allocation, geometric factors, Jacobi
// diagonals and the Chebyshev eigenvalue estimates (setup step of the hot path;
// the paper pre-computes its operators once at t = 0, Section 4.4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sem_internal.hpp"

namespace sem {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }
const char* last_error() { return g_err.c_str(); }

// First-appearance numbering of order-p triangle nodes: vertices by vertex id,
// edge nodes by (edge, position from the lower vertex id), interior nodes new.
void tri_numbering(int nvert, int ntri, const int* tri, int p, std::vector<int>& map2, long long& N2) {
    const int NT = (p + 1) * (p + 2) / 2;
    map2.assign((size_t)ntri * NT, -1);
    std::vector<long long> vid(nvert, -1);
    std::unordered_map<uint64_t, std::vector<long long>> edges;
    edges.reserve((size_t)ntri * 2);
    long long next = 0;
    for (int e = 0; e < ntri; ++e) {
        const int v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
        int n = 0;
        for (int j = 0; j <= p; ++j)
            for (int i = 0; i + j <= p; ++i, ++n) {
                long long* slot = nullptr;
                long long interior = -1;
                int vtx = -1;
                if (i == 0 && j == 0) vtx = v[0];
                else if (i == p && j == 0) vtx = v[1];
                else if (i == 0 && j == p) vtx = v[2];
                if (vtx >= 0) {
                    slot = &vid[vtx];
                } else {
                    int va = -1, vb = -1, pos = 0;
                    if (j == 0) { va = v[0]; vb = v[1]; pos = i; }
                    else if (i + j == p) { va = v[1]; vb = v[2]; pos = j; }
                    else if (i == 0) { va = v[2]; vb = v[0]; pos = p - j; }
                    if (va >= 0) {
                        if (va > vb) { std::swap(va, vb); pos = p - pos; }
                        const uint64_t key = ((uint64_t)(uint32_t)va << 32) | (uint32_t)vb;
                        auto& ids = edges[key];
                        if (ids.empty()) ids.assign(p - 1, -1);
                        slot = &ids[pos - 1];
                    } else {
                        slot = &interior;
                    }
                }
                if (*slot < 0) *slot = next++;
                map2[(size_t)e * NT + n] = (int)*slot;
            }
    }
    N2 = next;
}

// 2D coordinates of the order-p nodes (first appearance wins).
void tri_coords(int ntri, const int* tri, const double* vxy, int p, const std::vector<int>& map2, long long N2,
                std::vector<double>& xy) {
    const int NT = (p + 1) * (p + 2) / 2;
    const std::vector<double> tn = tri_nodes(p);
    xy.assign(2 * N2, 0.0);
    std::vector<char> seen(N2, 0);
    for (int e = 0; e < ntri; ++e) {
        const double* a = vxy + 2 * tri[3 * e];
        const double* b = vxy + 2 * tri[3 * e + 1];
        const double* c = vxy + 2 * tri[3 * e + 2];
        for (int n = 0; n < NT; ++n) {
            const int g = map2[(size_t)e * NT + n];
            if (seen[g]) continue;
            seen[g] = 1;
            const double r = tn[2 * n], s = tn[2 * n + 1];
            xy[2 * g] = -0.5 * (r + s) * a[0] + 0.5 * (1 + r) * b[0] + 0.5 * (1 + s) * c[0];
            xy[2 * g + 1] = -0.5 * (r + s) * a[1] + 0.5 * (1 + r) * b[1] + 0.5 * (1 + s) * c[1];
        }
    }
}

// Exact map of a base triangle with vertices v [3][2] at reference point (r, s): the affine
// map plus, for every curved edge f = (a, b) of arcs [3][3] (cx, cy, R; R = 0 straight), the
// displacement of the arc point from the chord times the blending factor 4 l_a l_b / (1 - xi^2),
// xi = l_b - l_a, l the barycentric coordinates (the triangle blending map of Szabo and
// Babuska).  The arc point lies at angle theta_a + (1 + xi)/2 (theta_b - theta_a), the angle
// difference taken the short way round.  The factor is one on the edge and zero on the two
// others; at the edge's end points it is 0/0 and the displacement is zero.
void blended_point(const double* v, const double* arcs, double r, double s, double* out) {
    const double lam[3] = {-0.5 * (r + s), 0.5 * (1.0 + r), 0.5 * (1.0 + s)};
    out[0] = lam[0] * v[0] + lam[1] * v[2] + lam[2] * v[4];
    out[1] = lam[0] * v[1] + lam[1] * v[3] + lam[2] * v[5];
    if (!arcs) return;
    static const int ends[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    for (int f = 0; f < 3; ++f) {
        const double cx = arcs[3 * f], cy = arcs[3 * f + 1], R = arcs[3 * f + 2];
        if (!(R > 0.0)) continue;
        const int a = ends[f][0], b = ends[f][1];
        const double xi = lam[b] - lam[a], den = 1.0 - xi * xi;
        if (!(den > 1e-13)) continue;
        const double ta = std::atan2(v[2 * a + 1] - cy, v[2 * a] - cx);
        const double tb = std::atan2(v[2 * b + 1] - cy, v[2 * b] - cx);
        const double dth = std::remainder(tb - ta, 2.0 * M_PI);
        const double th = ta + 0.5 * (1.0 + xi) * dth;
        const double px = cx + R * std::cos(th), py = cy + R * std::sin(th);
        const double qx = 0.5 * (1.0 - xi) * v[2 * a] + 0.5 * (1.0 + xi) * v[2 * b];
        const double qy = 0.5 * (1.0 - xi) * v[2 * a + 1] + 0.5 * (1.0 + xi) * v[2 * b + 1];
        const double fac = 4.0 * lam[a] * lam[b] / den;
        out[0] += fac * (px - qx);
        out[1] += fac * (py - qy);
    }
}

// The blended map of every base triangle at the order-p reference nodes, [ntri][NT][2].
void blended_nodes(int ntri, const int* tri, const double* vxy, const double* arc, int p, std::vector<double>& out) {
    const std::vector<double> tn = tri_nodes(p);
    const int NT = (p + 1) * (p + 2) / 2;
    out.assign((size_t)ntri * NT * 2, 0.0);
    for (int b = 0; b < ntri; ++b) {
        double v[6];
        for (int k = 0; k < 3; ++k) {
            v[2 * k] = vxy[2 * tri[3 * b + k]];
            v[2 * k + 1] = vxy[2 * tri[3 * b + k] + 1];
        }
        for (int n = 0; n < NT; ++n)
            blended_point(v, arc ? arc + 9 * (size_t)b : nullptr, tn[2 * n], tn[2 * n + 1], &out[((size_t)b * NT + n) * 2]);
    }
}

// 2D coordinates of the order-p nodes of a general mesh: the order-P geometry (node xy xyP
// [ntri][NT_P][2]) interpolated at the order-p nodes (first appearance wins).
void tri_coords_mapped(int ntri, int P, const std::vector<double>& xyP, int p, const std::vector<int>& map2,
                       long long N2, std::vector<double>& xy) {
    const int NT = (p + 1) * (p + 2) / 2, NTP = (P + 1) * (P + 2) / 2;
    std::vector<double> B, Dr, Ds;
    tri_lagrange(P, tri_nodes(p).data(), NT, B, Dr, Ds);
    xy.assign(2 * N2, 0.0);
    std::vector<char> seen(N2, 0);
    for (int e = 0; e < ntri; ++e)
        for (int n = 0; n < NT; ++n) {
            const int g = map2[(size_t)e * NT + n];
            if (seen[g]) continue;
            seen[g] = 1;
            double x = 0, y = 0;
            for (int k = 0; k < NTP; ++k) {
                x += B[(size_t)n * NTP + k] * xyP[((size_t)e * NTP + k) * 2];
                y += B[(size_t)n * NTP + k] * xyP[((size_t)e * NTP + k) * 2 + 1];
            }
            xy[2 * g] = x;
            xy[2 * g + 1] = y;
        }
}

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

template <typename T>
cudaError_t upload(T** p, const std::vector<T>& h) {
    cudaError_t e = dalloc(p, h.size());
    if (e != cudaSuccess) return e;
    if (!h.empty()) e = cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

std::vector<double> ref_block(const RefLevel& r) {
    // [Bt | Drt | Dst | BtT | DrT | DsT | Bz | Dz]
    std::vector<double> out;
    out.insert(out.end(), r.Bt.begin(), r.Bt.end());
    out.insert(out.end(), r.Drt.begin(), r.Drt.end());
    out.insert(out.end(), r.Dst.begin(), r.Dst.end());
    for (const std::vector<double>* M : {&r.Bt, &r.Drt, &r.Dst})
        for (int n = 0; n < r.NT; ++n)
            for (int q = 0; q < r.QT; ++q) out.push_back((*M)[(size_t)q * r.NT + n]);
    out.insert(out.end(), r.Bz.begin(), r.Bz.end());
    out.insert(out.end(), r.Dz.begin(), r.Dz.end());
    return out;
}

std::vector<float> to_float(const std::vector<double>& v) {
    std::vector<float> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
    return o;
}

}  // namespace

#define CK(expr)                                                                          \
    do {                                                                                  \
        cudaError_t _e = (expr);                                                          \
        if (_e != cudaSuccess) {                                                          \
            set_error(std::string("CUDA error in setup: ") + cudaGetErrorString(_e) +   \
                      " (" #expr ")");                                                    \
            return _e == cudaErrorMemoryAllocation ? SEM_ENOMEM : SEM_ECUDA;             \
        }                                                                                 \
    } while (0)

sem_status build_level(sem_handle* h, const sem_mesh* m, int li, int p, int pz) {
    Level& L = h->lv[li];
    L.dim = m->dim;
    L.p = p;
    L.pz = (m->dim == 3) ? pz : p;
    L.ref.build(m->dim, p, L.pz);
    L.NT = L.ref.NT; L.NZ = L.ref.NZ; L.QT = L.ref.QT; L.QZ = L.ref.QZ;
    L.Np = L.ref.Np; L.Nq = L.ref.Nq;
    L.ncomp = (m->dim == 3) ? 6 : 3;
    std::vector<int>& map2 = h->map2[li];
    long long N2 = 0;
    tri_numbering(m->nvert, m->ntri, m->tri, p, map2, N2);
    L.N2 = N2;
    const int nl = (m->dim == 3) ? m->nlayers : 1;
    L.E = (m->dim == 3) ? (int)h->elem_b.size() : m->ntri;
    L.N = (m->dim == 3) ? N2 * (long long)(nl * L.pz + 1) : N2;
    if (L.N >= (1LL << 31) - 1 || (long long)L.E * L.Np >= (1LL << 40)) {
        set_error("mesh too large for 32-bit node ids");
        return SEM_EINVAL;
    }
    std::vector<long long> gmap((size_t)L.E * L.Np);
    if (m->dim == 3) {
        for (size_t e = 0; e < (size_t)L.E; ++e) {
            const int b = h->elem_b[e], l = h->elem_l[e];
            for (int k = 0; k <= L.pz; ++k)
                for (int n = 0; n < L.NT; ++n)
                    gmap[e * L.Np + k * L.NT + n] = (long long)(l * L.pz + k) * N2 + map2[(size_t)b * L.NT + n];
        }
    } else {
        for (size_t i = 0; i < gmap.size(); ++i) gmap[i] = map2[i];
    }
    const int nf = (m->dim == 3) ? 5 : 3;
    std::vector<char> dmask(L.N, 0);
    for (int e = 0; e < L.E; ++e)
        for (int f = 0; f < nf; ++f)
            if (m->face_bc[(size_t)e * nf + f])
                for (int l : L.ref.face_nodes[f]) dmask[gmap[(size_t)e * L.Np + l]] = 1;
    {   // ids in no element (above a body): identity rows, listed with the Dirichlet nodes
        std::vector<char> held(L.N, 0);
        for (long long g : gmap) held[g] = 1;
        for (long long i = 0; i < L.N; ++i)
            if (!held[i]) dmask[i] = 1;
    }
    L.hdir.clear();
    for (long long i = 0; i < L.N; ++i)
        if (dmask[i]) L.hdir.push_back(i);
    if (L.hdir.empty()) {
        set_error("no Dirichlet face: the pure-Neumann Laplace problem is singular");
        return SEM_EINVAL;
    }
    L.hmap.resize(gmap.size());
    std::vector<int> mult(L.N, 0);
    std::vector<char> seen(L.N, 0);
    std::vector<unsigned char> owner(gmap.size(), 0);
    for (size_t i = 0; i < gmap.size(); ++i) {
        const long long g = gmap[i];
        L.hmap[i] = dmask[g] ? (int)(-g - 1) : (int)g;
        mult[g] += 1;
        if (!seen[g]) {
            seen[g] = 1;
            owner[i] = dmask[g] ? 0 : 1;
        }
    }
    std::vector<double> wm(L.N);
    for (long long i = 0; i < L.N; ++i) wm[i] = mult[i] > 0 ? 1.0 / mult[i] : 0.0;
    {   // +16 ints of padding: the tensor-core apply's bulk copies of the map round up to 16 B
        std::vector<int> padded(L.hmap);
        padded.resize(L.hmap.size() + 16, 0);
        CK(upload(&L.map, padded));
    }
    if (li == 0 && L.dim == 3) {   // elements that touch a Dirichlet node (the lifting apply's)
        std::vector<int> le;
        for (int e = 0; e < L.E; ++e)
            for (int l = 0; l < L.Np; ++l)
                if (L.hmap[(size_t)e * L.Np + l] < 0) { le.push_back(e); break; }
        L.nlift = (int)le.size();
        if (!le.empty()) CK(upload(&L.lift_elems, le));
    }
    CK(upload(&L.owner, owner));
    CK(upload(&L.wmult, wm));
    CK(upload(&L.wmult32, to_float(wm)));
    CK(upload(&L.dir, L.hdir));
    const std::vector<double> rb = ref_block(L.ref);
    CK(upload(&L.ref64.m, rb));
    CK(upload(&L.ref32.m, to_float(rb)));
    L.ref64.count = L.ref32.count = rb.size();
    CK(dalloc(&L.G, (size_t)L.E * L.ncomp * L.Nq));
    CK(dalloc(&L.G32, (size_t)L.E * L.ncomp * L.Nq + 16));   // +64 B: the tensor-core apply's bulk copies round up to 16 B
    CK(dalloc(&L.dinv, L.N));
    CK(dalloc(&L.dinv32, L.N));
    CK(dalloc(&L.u, L.N));
    CK(dalloc(&L.f, L.N));
    CK(dalloc(&L.y, L.N));
    CK(dalloc(&L.d, L.N));
    CK(dalloc(&L.u32, L.N));
    CK(dalloc(&L.f32, L.N));
    CK(dalloc(&L.y32, L.N));
    CK(dalloc(&L.d32, L.N));
    return SEM_OK;
}

// Geometric factors (FP64, FP32, BF16) of levels [first, last) from the handle's mesh and
// the order-P surface elevation h->eta2 (or a flat surface when `flat`).
sem_status geometry_levels(sem_handle* h, int first, int last, bool flat) {
    const int P = h->P;
    const Level& L0 = h->lv[0];
    const int ntri = (int)(h->tri.size() / 3);
    std::vector<double> vtri((size_t)ntri * 6);
    for (int b = 0; b < ntri; ++b)
        for (int k = 0; k < 3; ++k) {
            vtri[6 * b + 2 * k] = h->vxy[2 * h->tri[3 * b + k]];
            vtri[6 * b + 2 * k + 1] = h->vxy[2 * h->tri[3 * b + k] + 1];
        }
    double* dvtri = nullptr;
    CK(upload(&dvtri, vtri));
    const int NTP = L0.NT;
    std::vector<double> etaP((size_t)ntri * NTP, 0.0);
    if (!flat)
        for (int b = 0; b < ntri; ++b)
            for (int n = 0; n < NTP; ++n) etaP[(size_t)b * NTP + n] = h->eta2[h->map2[0][(size_t)b * NTP + n]];
    double* detaP = nullptr;
    CK(upload(&detaP, etaP));
    int *deb = nullptr, *del = nullptr;
    double *dxyP = nullptr, *dzif = nullptr;
    if (h->general) {
        CK(upload(&deb, h->elem_b));
        CK(upload(&del, h->elem_l));
        CK(upload(&dxyP, h->xyP));
        CK(upload(&dzif, h->zif));
    }
    for (int li = first; li < last; ++li) {
        Level& L = h->lv[li];
        std::vector<double> B, Dr, Ds;
        tri_lagrange(P, L.ref.tq.data(), L.QT, B, Dr, Ds);   // order-P map at level-p points
        double *dB = nullptr, *dDr = nullptr, *dDs = nullptr;
        CK(upload(&dB, B));
        CK(upload(&dDr, Dr));
        CK(upload(&dDs, Ds));
        cudaError_t e = h->general
                            ? launch_geometry_general(L, deb, del, dxyP, detaP, dzif, dB, dDr, dDs, NTP, 0)
                            : launch_geometry(L, dvtri, detaP, dB, dDr, dDs, NTP, h->nlayers, h->depth, 0);
        cudaFree(dB);
        cudaFree(dDr);
        cudaFree(dDs);
        CK(e);
        CK(build_g16(L, 0));
        CK(build_g16_t6(L, 0));
        if (L.Ae64 != nullptr) CK(element_matrices64(L, L.Ae64, 0));
        if (L.Adf != nullptr) CK(element_matrices_df(L, L.Adf, 0));
    }
    cudaFree(dvtri);
    cudaFree(detaP);
    if (h->general) {
        cudaFree(deb);
        cudaFree(del);
        cudaFree(dxyP);
        cudaFree(dzif);
    }
    return SEM_OK;
}

// Every layer of a mesh with given interfaces keeps a positive thickness at every order-P
// surface node: (a_{k+1} - a_k) + (b_{k+1} - b_k) eta > 0.
sem_status check_layers(const sem_handle* h, const std::vector<double>& eta) {
    if (!h->general || h->dim != 3) return SEM_OK;
    for (int k = 0; k < h->nlayers; ++k) {
        const double da = h->zif[2 * k + 2] - h->zif[2 * k], db = h->zif[2 * k + 3] - h->zif[2 * k + 1];
        for (double e : eta)
            if (!(da + db * e > 0.0)) {
                set_error("layer " + std::to_string(k) + " has no positive thickness at some surface node");
                return SEM_EINVAL;
            }
    }
    return SEM_OK;
}

sem_status build_geometry(sem_handle* h, const sem_mesh* m) {
    h->eta2.assign(h->lv[0].N2, 0.0);
    if (m->dim == 3 && m->eta) std::memcpy(h->eta2.data(), m->eta, sizeof(double) * h->lv[0].N2);
    const sem_status lay = check_layers(h, h->eta2);
    if (lay != SEM_OK) return lay;
    return geometry_levels(h, 0, (int)h->lv.size(), false);
}

// Assembled diagonal of level li and its inverse on the free nodes (FP64 and FP32).
sem_status diagonal_level(sem_handle* h, int li) {
    {
        Level& L = h->lv[li];
        double* dg = nullptr;
        CK(dalloc(&dg, L.N));
        CK(cudaMemset(dg, 0, sizeof(double) * L.N));
        CK(launch_diag(L, dg, 0));
        CK(cudaDeviceSynchronize());
        L.hdiag.resize(L.N);
        CK(cudaMemcpy(L.hdiag.data(), dg, sizeof(double) * L.N, cudaMemcpyDeviceToHost));
        cudaFree(dg);
        std::vector<double> dinv(L.N);
        std::vector<char> dm(L.N, 0);
        for (long long i : L.hdir) dm[i] = 1;
        for (long long i = 0; i < L.N; ++i) {
            if (!dm[i] && !(L.hdiag[i] > 0.0)) {
                set_error("non-positive diagonal entry: degenerate element");
                return SEM_EINVAL;
            }
            dinv[i] = dm[i] ? 0.0 : 1.0 / L.hdiag[i];
        }
        CK(cudaMemcpy(L.dinv, dinv.data(), sizeof(double) * L.N, cudaMemcpyHostToDevice));
        const std::vector<float> d32 = to_float(dinv);
        CK(cudaMemcpy(L.dinv32, d32.data(), sizeof(float) * L.N, cudaMemcpyHostToDevice));
    }
    return SEM_OK;
}

sem_status build_diagonals(sem_handle* h) {
    for (int li = 0; li < (int)h->lv.size(); ++li) {
        const sem_status st = diagonal_level(h, li);
        if (st != SEM_OK) return st;
    }
    return SEM_OK;
}

// Full reference gradients [dim][Nq][Np] of the coarsest level (thread-per-element apply
// inside the persistent coarse CG).
sem_status reassemble_coarse(sem_handle* h);

sem_status build_coarse_gradients(sem_handle* h) {
    Level& C = h->lv.back();
    const RefLevel& r = C.ref;
    std::vector<double> g((size_t)C.dim * C.Nq * C.Np);
    for (int qz = 0; qz < C.QZ; ++qz)
        for (int qt = 0; qt < C.QT; ++qt)
            for (int k = 0; k < C.NZ; ++k)
                for (int n = 0; n < C.NT; ++n) {
                    const int q = qz * C.QT + qt, l = k * C.NT + n;
                    const double bz = r.Bz[qz * C.NZ + k], dz = r.Dz[qz * C.NZ + k];
                    g[(size_t)(0 * C.Nq + q) * C.Np + l] = r.Drt[qt * C.NT + n] * bz;
                    g[(size_t)(1 * C.Nq + q) * C.Np + l] = r.Dst[qt * C.NT + n] * bz;
                    if (C.dim == 3) g[(size_t)(2 * C.Nq + q) * C.Np + l] = r.Bt[qt * C.NT + n] * dz;
                }
    CK(upload(&C.gref, g));
    // CSR pattern of the free-free coarse matrix and the slot of every element entry
    if ((long long)C.E * C.Np * C.Np > (1LL << 28)) return SEM_OK;   // large coarse elements: matrix-free CG
    std::vector<std::vector<int>> cols(C.N);
    for (int e = 0; e < C.E; ++e)
        for (int i = 0; i < C.Np; ++i) {
            const int gi = C.hmap[(size_t)e * C.Np + i];
            if (gi < 0) continue;
            for (int j = 0; j < C.Np; ++j) {
                const int gj = C.hmap[(size_t)e * C.Np + j];
                if (gj >= 0) cols[gi].push_back(gj);
            }
        }
    std::vector<int> rowptr(C.N + 1, 0), col;
    for (long long i = 0; i < C.N; ++i) {
        std::sort(cols[i].begin(), cols[i].end());
        cols[i].erase(std::unique(cols[i].begin(), cols[i].end()), cols[i].end());
        rowptr[i + 1] = rowptr[i] + (int)cols[i].size();
        col.insert(col.end(), cols[i].begin(), cols[i].end());
    }
    std::vector<int> slot((size_t)C.E * C.Np * C.Np, -1);
    for (int e = 0; e < C.E; ++e)
        for (int i = 0; i < C.Np; ++i) {
            const int gi = C.hmap[(size_t)e * C.Np + i];
            if (gi < 0) continue;
            for (int j = 0; j < C.Np; ++j) {
                const int gj = C.hmap[(size_t)e * C.Np + j];
                if (gj < 0) continue;
                const auto it = std::lower_bound(cols[gi].begin(), cols[gi].end(), gj);
                slot[((size_t)e * C.Np + i) * C.Np + j] = rowptr[gi] + (int)(it - cols[gi].begin());
            }
        }
    C.csr_nnz = (long long)col.size();
    CK(upload(&C.csr_rowptr, rowptr));
    CK(upload(&C.csr_col, col));
    CK(upload(&C.csr_slot, slot));          // kept: the values are reassembled when eta changes
    CK(dalloc(&C.csr_val, col.size()));
    if (h->opts.deterministic) {
        // every CSR entry sums its element entries in a fixed (ascending) order: the entry ->
        // element-entry map by a counting sort over slot
        std::vector<int> eptr((size_t)C.csr_nnz + 1, 0);
        for (size_t t = 0; t < slot.size(); ++t)
            if (slot[t] >= 0) ++eptr[(size_t)slot[t] + 1];
        for (long long k = 0; k < C.csr_nnz; ++k) eptr[(size_t)k + 1] += eptr[(size_t)k];
        std::vector<int> fill(eptr.begin(), eptr.end() - 1), eidx((size_t)eptr[(size_t)C.csr_nnz]);
        for (size_t t = 0; t < slot.size(); ++t)
            if (slot[t] >= 0) eidx[(size_t)fill[(size_t)slot[t]]++] = (int)t;
        CK(upload(&C.csr_eptr, eptr));
        CK(upload(&C.csr_eidx, eidx));
        CK(dalloc(&C.csr_ev, slot.size()));
        CK(cudaMemset(C.csr_ev, 0, sizeof(double) * slot.size()));
    }
    return reassemble_coarse(h);
}

// Recursive coordinate bisection of idx[lo, hi) into `parts` contiguous runs (the longer extent
// of the first two coordinates is cut, in proportion to the parts on each side; xyz holds `st`
// coordinates per node, the third, if any, breaks ties); ptr gets the run ends.
void rcb_split(std::vector<int>& idx, int lo, int hi, int parts, const std::vector<double>& xyz, int st,
               std::vector<int>& ptr) {
    if (parts <= 1 || hi - lo <= 1) {
        ptr.push_back(hi);
        return;
    }
    double mn[2] = {1e300, 1e300}, mx[2] = {-1e300, -1e300};
    for (int i = lo; i < hi; ++i)
        for (int a = 0; a < 2; ++a) {
            mn[a] = std::min(mn[a], xyz[st * (size_t)idx[i] + a]);
            mx[a] = std::max(mx[a], xyz[st * (size_t)idx[i] + a]);
        }
    const int ax = (mx[1] - mn[1] > mx[0] - mn[0]) ? 1 : 0;
    std::stable_sort(idx.begin() + lo, idx.begin() + hi, [&](int a, int b) {
        const double va = xyz[st * (size_t)a + ax], vb = xyz[st * (size_t)b + ax];
        return va < vb || (va == vb && st > 2 && xyz[st * (size_t)a + 2] < xyz[st * (size_t)b + 2]);
    });
    const int p1 = parts / 2;
    const int cut = lo + (int)std::llround((double)(hi - lo) * p1 / parts);
    rcb_split(idx, lo, cut, p1, xyz, st, ptr);
    rcb_split(idx, cut, hi, parts - p1, xyz, st, ptr);
}

// Inverse of the SPD matrix a (n x n, row major) by Cholesky, in place; false if a pivot is
// not positive.
bool spd_inverse(std::vector<double>& a, int n) {
    for (int j = 0; j < n; ++j) {                       // a = L L^T, L in the lower triangle
        double d = a[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        a[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = a[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
            a[(size_t)i * n + j] = v / d;
        }
    }
    std::vector<double> li((size_t)n * n, 0.0);        // L^{-1}, lower triangular
    for (int j = 0; j < n; ++j) {
        li[(size_t)j * n + j] = 1.0 / a[(size_t)j * n + j];
        for (int i = j + 1; i < n; ++i) {
            double v = 0.0;
            for (int k = j; k < i; ++k) v -= a[(size_t)i * n + k] * li[(size_t)k * n + j];
            li[(size_t)i * n + j] = v / a[(size_t)i * n + i];
        }
    }
    for (int i = 0; i < n; ++i)                         // A^{-1} = L^{-T} L^{-1}, symmetric
        for (int j = 0; j <= i; ++j) {
            double v = 0.0;
            for (int k = i; k < n; ++k) v += li[(size_t)k * n + i] * li[(size_t)k * n + j];
            a[(size_t)i * n + j] = a[(size_t)j * n + i] = v;
        }
    return true;
}

// Block-Jacobi preconditioner of the coarse CG (sem_options.coarse_bj): the free rows cut into
// patches of at most kBjMax (about 120) by coordinate bisection, once; the FP32 inverse of each
// patch's diagonal block from the current coarse matrix, every time it is reassembled.
sem_status build_coarse_bj(sem_handle* h) {
    Level& C = h->lv.back();
    if (!h->opts.coarse_bj || h->opts.batch != 0 || C.csr_val == nullptr) return SEM_OK;
    const long long N = C.N;
    std::vector<int> rowptr(N + 1), col((size_t)C.csr_nnz);
    std::vector<double> val((size_t)C.csr_nnz);
    CK(cudaMemcpy(rowptr.data(), C.csr_rowptr, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(col.data(), C.csr_col, sizeof(int) * col.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(val.data(), C.csr_val, sizeof(double) * val.size(), cudaMemcpyDeviceToHost));
    if (C.hbj_ptr.empty()) {
        std::vector<int> freer;
        for (long long i = 0; i < N; ++i)
            if (rowptr[i + 1] > rowptr[i]) freer.push_back((int)i);
        const int nf = (int)freer.size();
        const int nb = (nf + 119) / 120;
        if (nf == 0) return SEM_OK;
        std::vector<double> xyz(3 * (size_t)N);
        const sem_status cst = sem_node_coords(h, (int)h->lv.size() - 1, xyz.data());
        if (cst != SEM_OK) return cst;
        std::vector<int> ptr{0};
        rcb_split(freer, 0, nf, nb, xyz, h->dim == 3 ? 3 : 2, ptr);   // 2D: (x, z) per node
        int nnzmax = 0;
        for (size_t b = 0; b + 1 < ptr.size(); ++b) {
            if (ptr[b + 1] - ptr[b] > kBjMax) return SEM_OK;               // point-Jacobi CG
            int nnz = 0;
            for (int k = ptr[b]; k < ptr[b + 1]; ++k) nnz += rowptr[freer[k] + 1] - rowptr[freer[k]];
            nnzmax = std::max(nnzmax, nnz);
        }
        if (nb > coarse_bj_capacity(nnzmax)) return SEM_OK;               // point-Jacobi CG
        std::vector<int> lptr((ptr.size() - 1) * (kBjMax + 1), 0), lidx((ptr.size() - 1) * (size_t)nnzmax, 0);
        for (size_t b = 0; b + 1 < ptr.size(); ++b) {
            int acc = 0;
            for (int k = ptr[b]; k < ptr[b + 1]; ++k) {
                lptr[b * (kBjMax + 1) + (k - ptr[b])] = acc;
                for (int a = rowptr[freer[k]]; a < rowptr[freer[k] + 1]; ++a) lidx[b * (size_t)nnzmax + acc++] = a;
            }
            lptr[b * (kBjMax + 1) + (ptr[b + 1] - ptr[b])] = acc;
        }
        C.bj_nnzmax = nnzmax;
        C.hbj_ptr = ptr;
        C.hbj_rows = freer;
        CK(upload(&C.bj_ptr, ptr));
        CK(upload(&C.bj_rows, freer));
        CK(upload(&C.bj_lptr, lptr));
        CK(upload(&C.bj_lidx, lidx));
        CK(dalloc(&C.bj_inv, (size_t)(ptr.size() - 1) * kBjMax * kBjMax));
    }
    const int nb = (int)C.hbj_ptr.size() - 1;
    std::vector<float> inv((size_t)nb * kBjMax * kBjMax, 0.f);
    std::vector<char> ok(nb, 1);
    auto work = [&](int b0, int b1) {
        for (int b = b0; b < b1; ++b) {
            const int k0 = C.hbj_ptr[b], n = C.hbj_ptr[b + 1] - k0;
            std::unordered_map<int, int> loc;
            for (int k = 0; k < n; ++k) loc[C.hbj_rows[k0 + k]] = k;
            std::vector<double> a((size_t)n * n, 0.0);
            for (int k = 0; k < n; ++k) {
                const int row = C.hbj_rows[k0 + k];
                for (int t = rowptr[row]; t < rowptr[row + 1]; ++t) {
                    const auto it = loc.find(col[t]);
                    if (it != loc.end()) a[(size_t)k * n + it->second] = val[t];
                }
            }
            for (int i = 0; i < n; ++i)                 // the assembled block, symmetrised
                for (int j = 0; j < i; ++j)
                    a[(size_t)i * n + j] = a[(size_t)j * n + i] = 0.5 * (a[(size_t)i * n + j] + a[(size_t)j * n + i]);
            if (!spd_inverse(a, n)) { ok[b] = 0; continue; }
            float* dst = inv.data() + (size_t)b * kBjMax * kBjMax;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) dst[(size_t)i * kBjMax + j] = (float)a[(size_t)i * n + j];
        }
    };
    const int nt = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(work, (int)((long long)nb * t / nt), (int)((long long)nb * (t + 1) / nt));
    for (std::thread& th : pool) th.join();
    for (int b = 0; b < nb; ++b)
        if (!ok[b]) {
            set_error("coarse block-Jacobi: a diagonal block is not positive definite");
            return SEM_BREAKDOWN;
        }
    CK(cudaMemcpy(C.bj_inv, inv.data(), sizeof(float) * inv.size(), cudaMemcpyHostToDevice));
    C.bj_nb = nb;
    return SEM_OK;
}

// Values of the assembled coarse matrix from the coarsest level's current geometric factors,
// and the block-Jacobi inverses that depend on them.
sem_status reassemble_coarse(sem_handle* h) {
    Level& C = h->lv.back();
    if (C.csr_val == nullptr) return SEM_OK;
    CK(cudaMemset(C.csr_val, 0, sizeof(double) * C.csr_nnz));
    CK(coarse_assemble(C, C.gref, C.csr_slot, C.csr_val, 0));    // atomic, or fixed-order sums (deterministic)
    CK(cudaDeviceSynchronize());
    return build_coarse_bj(h);
}

sem_status build_transfers(sem_handle* h) {
    for (size_t li = 0; li + 1 < h->lv.size(); ++li) {
        Level& F = h->lv[li];
        const Level& C = h->lv[li + 1];
        std::vector<double> Bt, Bz;
        interp_factors(F.dim, F.p, C.p, F.pz, C.pz, Bt, Bz);
        CK(upload(&F.It64, Bt));
        CK(upload(&F.Iz64, Bz));
        CK(upload(&F.It32, to_float(Bt)));
        CK(upload(&F.Iz32, to_float(Bz)));
    }
    return SEM_OK;
}

// Surface operators and work fields of the free-surface time stepping (surface_ops = 1):
// the order-P surface is the top of the top sigma layer and must be exactly the Dirichlet set.
sem_status build_surface(sem_handle* h) {
    if (h->dim != 3 || h->general) { set_error("surface_ops needs a 3D sigma-layer mesh"); return SEM_EINVAL; }
    const Level& L0 = h->lv[0];
    const long long N2 = L0.N2, k_top = (long long)h->nlayers * L0.pz;
    bool top_only = (long long)L0.hdir.size() == N2;
    for (long long i = 0; top_only && i < N2; ++i) top_only = L0.hdir[i] == k_top * N2 + i;
    if (!top_only) {
        set_error("surface_ops: the Dirichlet nodes must be exactly the free-surface nodes");
        return SEM_EINVAL;
    }
    const int ntri = (int)(h->tri.size() / 3), NT = L0.NT;
    std::vector<double> vtri((size_t)ntri * 6);
    for (int b = 0; b < ntri; ++b)
        for (int k = 0; k < 3; ++k) {
            vtri[6 * b + 2 * k] = h->vxy[2 * h->tri[3 * b + k]];
            vtri[6 * b + 2 * k + 1] = h->vxy[2 * h->tri[3 * b + k] + 1];
        }
    std::vector<double> B, Dr, Ds, Bz, Dz;
    tri_lagrange(h->P, L0.ref.tnodes.data(), NT, B, Dr, Ds);        // derivatives at the nodes
    const double one = 1.0;
    lagrange1d(L0.ref.znodes, &one, 1, Bz, Dz);                      // h_k'(+1)
    std::vector<double> mult(N2, 0.0);
    for (size_t i = 0; i < h->map2[0].size(); ++i) mult[h->map2[0][i]] += 1.0;
    for (double& m : mult) m = m > 0 ? 1.0 / m : 0.0;
    CK(upload(&h->fs_map2, h->map2[0]));
    CK(upload(&h->fs_vtri, vtri));
    CK(upload(&h->fs_Drn, Dr));
    CK(upload(&h->fs_Dsn, Ds));
    CK(upload(&h->fs_Dtop, Dz));
    CK(upload(&h->fs_invm, mult));
    CK(upload(&h->fs_eta, h->eta2));
    CK(dalloc(&h->fs_phi, L0.N));
    for (double** v : {&h->fs_w, &h->fs_ex, &h->fs_ey, &h->fs_px, &h->fs_py, &h->fs_se, &h->fs_sp}) CK(dalloc(v, N2));
    CK(dalloc(&h->fs_k, 8 * N2));
    CK(cudaMallocHost((void**)&h->fs_hpin, sizeof(double) * N2));
    return SEM_OK;
}

sem_status build_workspace(sem_handle* h) {
    const long long N = h->lv[0].N;
    const Level& Lc = h->lv.back();
    Scratch& sc = h->sc;
    CK(dalloc(&sc.part, (size_t)reduce_blocks() * 66));
    CK(dalloc(&sc.counter, 4));
    CK(cudaMemset(sc.counter, 0, 4 * sizeof(unsigned)));
    CK(dalloc(&sc.scal, 128));
    CK(cudaMemset(sc.scal, 0, 128 * sizeof(double)));
    CK(dalloc(&sc.flags, kFlagCount));
    CK(cudaMemset(sc.flags, 0, kFlagCount * sizeof(int)));
    h->net.err = sc.flags + F_TC_ERR;          // the network's tensor-core GEMMs report on the same flag
    for (Level& L : h->lv) L.df_err = sc.flags + F_TC_ERR;     // and the double-FP32 apply's tile copies
    CK(cudaMallocHost((void**)&sc.hpinned, 128 * sizeof(double)));
    CK(cudaMallocHost((void**)&sc.hflags, kFlagCount * sizeof(int)));
    for (double** v : {&h->r, &h->z, &h->p, &h->q, &h->x, &h->fr}) CK(dalloc(v, N));
    if (h->opts.outer == SEM_OUTER_FGMRES) {
        CK(dalloc(&h->V, (size_t)(h->opts.gmres_m + 1) * N));
        CK(dalloc(&h->Zb, (size_t)h->opts.gmres_m * N));
        CK(dalloc(&h->gm_y, (size_t)h->opts.gmres_m));
    }
    for (double** v : {&h->cx, &h->cr, &h->cz, &h->cp, &h->cq, &h->cb}) CK(dalloc(v, Lc.N));
    if (h->opts.precision != SEM_PREC_FP64 && h->opts.inner_imax > 0)
        for (float** v : {&h->ir, &h->iz, &h->ip, &h->iq, &h->ie}) CK(dalloc(v, N));
    if (h->opts.batch) {
        CK(dalloc(&h->bu, N));
        CK(cudaStreamCreateWithFlags(&h->bstream, cudaStreamNonBlocking));
    }
    CK(dalloc(&h->st_eta, h->lv[0].hdir.size()));
    CK(dalloc(&h->st_rhs, N));
    CK(dalloc(&h->st_phi, N));
    if (h->opts.surface_ops) {
        const sem_status st = build_surface(h);
        if (st != SEM_OK) return st;
    }
    if (h->opts.profile) {
        h->ev.resize(512);
        h->ev_kind.assign(256, 0);
        for (auto& e : h->ev) CK(cudaEventCreate(&e));
    }
    return SEM_OK;
}

// Correction network, its Adam state and the buffers of the learned sweep and its
// training (finest level), allocated when smoother = LEARNED.  Initial weights:
// Glorot-uniform W1, W2 scaled by 0.1 (a small first correction), zero biases.
sem_status build_mlp(sem_handle* h) {
    if (h->opts.smoother != SEM_SMOOTH_LEARNED) return SEM_OK;
    const Level& L = h->lv[0];
    MlpNet& n = h->net;
    n.nin = n.nout = L.Np;
    n.H = h->opts.mlp_hidden;
    const size_t n1 = (size_t)n.H * n.nin, n2 = (size_t)n.nout * n.H;
    std::mt19937_64 rng(h->opts.mlp_seed);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    const double a1 = std::sqrt(6.0 / (n.nin + n.H)), a2 = 0.1 * std::sqrt(6.0 / (n.nout + n.H));
    std::vector<float> W1(n1), W2(n2), b1(n.H, 0.f), b2(n.nout, 0.f);
    for (auto& w : W1) w = (float)(a1 * U(rng));
    for (auto& w : W2) w = (float)(a2 * U(rng));
    CK(upload(&n.W1, W1));
    CK(upload(&n.W2, W2));
    CK(upload(&n.b1, b1));
    CK(upload(&n.b2, b2));
    CK(dalloc(&n.W1b, n1));
    CK(dalloc(&n.W2b, n2));
    CK(mlp_sync_bf16(n, 0));
    MlpGrads& g = h->grads;
    CK(dalloc(&g.dW1, n1));
    CK(dalloc(&g.dW2, n2));
    CK(dalloc(&g.db1, n.H));
    CK(dalloc(&g.db2, n.nout));
    const size_t sizes[4] = {n1, (size_t)n.H, n2, (size_t)n.nout};
    for (int k = 0; k < 4; ++k) {
        CK(dalloc(&h->adam.m[k], sizes[k]));
        CK(dalloc(&h->adam.v[k], sizes[k]));
        CK(cudaMemset(h->adam.m[k], 0, sizeof(float) * sizes[k]));
        CK(cudaMemset(h->adam.v[k], 0, sizeof(float) * sizes[k]));
    }
    const size_t ep = (size_t)L.E * L.Np, eh = (size_t)L.E * n.H;
    for (float** v : {&h->mX, &h->mT, &h->mY, &h->mdY}) CK(dalloc(v, ep));
    for (float** v : {&h->mA1, &h->mH1, &h->mdH}) CK(dalloc(v, eh));
    CK(dalloc(&h->mscale, L.E));
    for (float** v : {&h->lr32, &h->ld32, &h->lu32, &h->te0, &h->tf, &h->tu, &h->tz}) CK(dalloc(v, L.N));
    CK(cudaDeviceSynchronize());
    return SEM_OK;
}

}  // namespace sem
