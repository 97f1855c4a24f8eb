// GPU construction of the S-EFIE H-Matrix from a triangle mesh
// (arxiv 2307.03968 §II eqs. 3-5), the plane-wave excitation of both bases,
// and the dispatch of hm_build by basis.
//
// Host (C++): RWG basis; the tree, partition and layout are the shared ones
// of k_assemble.cuh.  Device: the Galerkin RWG entry (eq. 3 tested with RWG
// functions) used by the shared fill and ACA kernels.
//
// Discretisation (the paper is silent on it; the same choices as the
// documented reading of the whole build): time convention e^{jwt},
// G = exp(-jkR)/(4 pi R), 7-point degree-5 triangle rule, and for triangle
// pairs whose centroids are closer than 2 x the larger maximum edge length the
// 1/R part of G is integrated analytically over the source triangle (Wilton et
// al. 1984 / Graglia 1993 potential integrals) with only the smooth remainder
// on the quadrature points.
#include "k_assemble.cuh"

namespace hm {
namespace {

constexpr int NQ = 7;
constexpr double EXTRACT_FACTOR = 2.0;

// ---------------------------------------------------------------- geometry ----
struct Geo {
    const double *vtx;    // nv x 3
    const int32_t *tri;   // nt x 3
    const double *cen;    // nt x 3 centroids
    const double *hmax;   // nt max edge length
    const double *area;   // nt
    const double *nrm;    // nt x 3 unit normal
    const double *qpd;    // nt x NQ x 3 quadrature points
    const int32_t *etri;  // ne x 2 (T+, T-)
    const int32_t *efree; // ne x 2
    const double *elen;   // ne
    const int32_t *perm;  // tree position -> original edge index
    double k, eta;
    template <class R> __device__ CX<R> entry(int m, int n) const;
};

__constant__ double c_qw[NQ];

// The singular-extraction predicate, evaluated in FP64 without contractions so
// that it takes the same decision as any other IEEE FP64 evaluation of
// |c_m - c_n|^2 < (2 h)^2.
__device__ __forceinline__ bool extract_pair(const Geo &g, int tm, int tn)
{
    const double dx = __dsub_rn(g.cen[3 * tm], g.cen[3 * tn]);
    const double dy = __dsub_rn(g.cen[3 * tm + 1], g.cen[3 * tn + 1]);
    const double dz = __dsub_rn(g.cen[3 * tm + 2], g.cen[3 * tn + 2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double h = g.hmax[tm] > g.hmax[tn] ? g.hmax[tm] : g.hmax[tn];
    const double lim = __dmul_rn(EXTRACT_FACTOR, h);
    return d2 < __dmul_rn(lim, lim);
}

// Int_T 1/R dS' (s0) and Int_T (rho' - rho)/R dS' (s1, in-plane) for the flat
// triangle tn and observation point r (coordinates relative to vertex p0).
template <class R>
__device__ void potential(const Geo &g, int tn, const R r[3], R &s0, R s1[3])
{
    const int32_t *tv = g.tri + 3 * tn;
    R P[3][3];
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) P[a][d] = (R)(g.vtx[3 * tv[a] + d] - g.vtx[3 * tv[0] + d]);
    R n[3];
    for (int d = 0; d < 3; ++d) n[d] = (R)g.nrm[3 * tn + d];
    const R dd = n[0] * r[0] + n[1] * r[1] + n[2] * r[2];
    const R ad = absR(dd);
    const R rho[3] = {r[0] - dd * n[0], r[1] - dd * n[1], r[2] - dd * n[2]};
    s0 = 0;
    s1[0] = s1[1] = s1[2] = 0;
    for (int e = 0; e < 3; ++e) {
        const R *a = P[e], *b = P[(e + 1) % 3];
        R lv[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const R ll = sqrtR(lv[0] * lv[0] + lv[1] * lv[1] + lv[2] * lv[2]);
        const R lh[3] = {lv[0] / ll, lv[1] / ll, lv[2] / ll};
        const R uh[3] = {lh[1] * n[2] - lh[2] * n[1], lh[2] * n[0] - lh[0] * n[2], lh[0] * n[1] - lh[1] * n[0]};
        const R am[3] = {a[0] - rho[0], a[1] - rho[1], a[2] - rho[2]};
        const R bm[3] = {b[0] - rho[0], b[1] - rho[1], b[2] - rho[2]};
        const R lp = bm[0] * lh[0] + bm[1] * lh[1] + bm[2] * lh[2];
        const R lm = am[0] * lh[0] + am[1] * lh[1] + am[2] * lh[2];
        const R t = am[0] * uh[0] + am[1] * uh[1] + am[2] * uh[2];
        const R R02 = t * t + dd * dd;
        const R Rp = sqrtR(R02 + lp * lp), Rm = sqrtR(R02 + lm * lm);
        R f = 0;
        if (R02 > 0) f = (lm < 0 && lp < 0) ? logR((Rm - lm) / (Rp - lp)) : logR((Rp + lp) / (Rm + lm));
        if (R02 > 0) {
            R term = t * f;
            if (ad > 0) term -= ad * (atanR(t * lp / (R02 + ad * Rp)) - atanR(t * lm / (R02 + ad * Rm)));
            s0 += term;
        }
        const R gg = (R)0.5 * ((R02 > 0 ? R02 * f : (R)0) + lp * Rp - lm * Rm);
        s1[0] += gg * uh[0];
        s1[1] += gg * uh[1];
        s1[2] += gg * uh[2];
    }
}

// (1/(A_m A_n)) Int_Tm Int_Tn [ 1/4 (r - vm).(r' - vn) - 1/k^2 ] G dS' dS
// Coordinates are taken relative to vertex 0 of tn to keep FP32 accurate.
template <class R>
__device__ CX<R> pair_integral(const Geo &g, int tm, int vmi, int tn, int vni)
{
    const R k = (R)g.k, ik2 = (R)(1.0 / (g.k * g.k));
    const R inv4pi = (R)(0.25 / 3.14159265358979323846);
    const bool extract = extract_pair(g, tm, tn);
    const double *o = g.vtx + 3 * g.tri[3 * tn];
    const R vm[3] = {(R)(g.vtx[3 * vmi] - o[0]), (R)(g.vtx[3 * vmi + 1] - o[1]), (R)(g.vtx[3 * vmi + 2] - o[2])};
    const R vn[3] = {(R)(g.vtx[3 * vni] - o[0]), (R)(g.vtx[3 * vni + 1] - o[1]), (R)(g.vtx[3 * vni + 2] - o[2])};
    R qn[NQ][3];
    for (int j = 0; j < NQ; ++j)
        for (int d = 0; d < 3; ++d) qn[j][d] = (R)(g.qpd[(tn * NQ + j) * 3 + d] - o[d]);
    CX<R> acc{0, 0};
    for (int i = 0; i < NQ; ++i) {
        R ri[3];
        for (int d = 0; d < 3; ++d) ri[d] = (R)(g.qpd[(tm * NQ + i) * 3 + d] - o[d]);
        const R a[3] = {ri[0] - vm[0], ri[1] - vm[1], ri[2] - vm[2]};
        CX<R> inner{0, 0};
        for (int j = 0; j < NQ; ++j) {
            const R bj[3] = {qn[j][0] - vn[0], qn[j][1] - vn[1], qn[j][2] - vn[2]};
            const R dr[3] = {ri[0] - qn[j][0], ri[1] - qn[j][1], ri[2] - qn[j][2]};
            const R Rr = sqrtR(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
            const R fac = (R)0.25 * (a[0] * bj[0] + a[1] * bj[1] + a[2] * bj[2]) - ik2;
            R gre, gim;
            if (extract) {
                if (Rr < (R)1e-12) { gre = 0; gim = -k * inv4pi; }
                else {
                    const R sh = sinR((R)0.5 * k * Rr);
                    gre = -(R)2 * sh * sh * inv4pi / Rr;
                    gim = -sinR(k * Rr) * inv4pi / Rr;
                }
            } else {
                R s, c;
                sincosR(k * Rr, &s, &c);
                gre = c * inv4pi / Rr;
                gim = -s * inv4pi / Rr;
            }
            const R w = (R)c_qw[j] * fac;
            inner.re += w * gre;
            inner.im += w * gim;
        }
        if (extract) {
            R s0, s1[3];
            potential<R>(g, tn, ri, s0, s1);
            const R nx = (R)g.nrm[3 * tn], ny = (R)g.nrm[3 * tn + 1], nz = (R)g.nrm[3 * tn + 2];
            const R dd = nx * ri[0] + ny * ri[1] + nz * ri[2];
            const R rv[3] = {ri[0] - dd * nx - vn[0], ri[1] - dd * ny - vn[1], ri[2] - dd * nz - vn[2]};
            const R S1[3] = {s1[0] + rv[0] * s0, s1[1] + rv[1] * s0, s1[2] + rv[2] * s0};
            inner.re += ((R)0.25 * (a[0] * S1[0] + a[1] * S1[1] + a[2] * S1[2]) - ik2 * s0) * inv4pi /
                        (R)g.area[tn];
        }
        acc.re += (R)c_qw[i] * inner.re;
        acc.im += (R)c_qw[i] * inner.im;
    }
    return acc;
}

// Z[m][n] for original RWG indices m, n
template <class R>
__device__ CX<R> rwg_entry(const Geo &g, int m, int n)
{
    CX<R> z{0, 0};
    for (int p = 0; p < 2; ++p) {
        const int tm = g.etri[2 * m + p], vm = g.efree[2 * m + p];
        for (int q = 0; q < 2; ++q) {
            const int tn = g.etri[2 * n + q], vn = g.efree[2 * n + q];
            const CX<R> v = pair_integral<R>(g, tm, vm, tn, vn);
            const R s = (p == q) ? (R)1 : (R)-1;
            z.re += s * v.re;
            z.im += s * v.im;
        }
    }
    // multiply by j k eta l_m l_n
    const R f = (R)(g.k * g.eta * g.elen[m] * g.elen[n]);
    return CX<R>{-f * z.im, f * z.re};
}

template <class R> __device__ CX<R> Geo::entry(int m, int n) const { return rwg_entry<R>(*this, m, n); }


// b[r*ldb + m] = sum_s ucoef[m][s] sum_q w_q (r_q - v_s) . p_hat exp(-jk k_hat . r_q): the
// Galerkin projection of a unit plane wave on RWG (7-point rule per triangle,
// ucoef = +-l/2) or kappa-weighted SWG functions (4-point rule per
// tetrahedron, ucoef = +-kappa a / 3)
__global__ void k_rhs_plane_wave(const double *__restrict__ qpd, const double *__restrict__ qw, int nq,
                                 const double *__restrict__ vtx, const int32_t *__restrict__ ucell,
                                 const int32_t *__restrict__ ufree, const double *__restrict__ ucoef, int64_t N,
                                 double k, const double *__restrict__ kh, const double *__restrict__ ph, int nrhs,
                                 float2 *b, int64_t ldb)
{
    const int64_t total = N * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / N, m = t - r * N;
        const double *kk = kh + 3 * r, *pp = ph + 3 * r;
        double re = 0.0, im = 0.0;
        for (int p = 0; p < 2; ++p) {
            const int c = ucell[2 * m + p];
            if (c < 0) continue;
            const double *v = vtx + 3 * ufree[2 * m + p];
            double sre = 0.0, sim = 0.0;
            for (int q = 0; q < nq; ++q) {
                const double *rq = qpd + ((int64_t)c * nq + q) * 3;
                const double proj = (rq[0] - v[0]) * pp[0] + (rq[1] - v[1]) * pp[1] + (rq[2] - v[2]) * pp[2];
                double sn, cs;
                sincos(k * (kk[0] * rq[0] + kk[1] * rq[1] + kk[2] * rq[2]), &sn, &cs);
                sre += qw[q] * proj * cs;
                sim -= qw[q] * proj * sn;
            }
            re += ucoef[2 * m + p] * sre;
            im += ucoef[2 * m + p] * sim;
        }
        b[r * ldb + m] = make_float2((float)re, (float)im);
    }
}

// RWG edges: interior edges sorted by (min vertex, max vertex), T+ = lower triangle
struct RwgEdges {
    std::vector<int32_t> etri, efree;   // N x 2
    std::vector<int64_t> ev;            // N x 2 vertex ids
};

hm_status rwg_edges(const hm_mesh *mesh, RwgEdges &E)
{
    const int64_t nv = mesh->n_vert, nt = mesh->n_cell;
    if (nv < 3 || nt < 2 || !mesh->xyz || !mesh->cells) return fail(HM_ERR_ARG, "empty mesh");
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (mesh->cells[i] < 0 || mesh->cells[i] >= nv) return fail(HM_ERR_ARG, "triangle vertex id out of range");
    struct HE { int64_t key; int32_t t, w; };
    std::vector<HE> he;
    he.reserve(3 * nt);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *v = mesh->cells + 3 * t;
        for (int e = 0; e < 3; ++e) {
            const int32_t a = v[e], b = v[(e + 1) % 3], w = v[(e + 2) % 3];
            const int64_t lo = std::min(a, b), hi = std::max(a, b);
            he.push_back({lo * nv + hi, (int32_t)t, w});
        }
    }
    std::sort(he.begin(), he.end(), [](const HE &x, const HE &y) { return x.key < y.key || (x.key == y.key && x.t < y.t); });
    for (size_t i = 0; i < he.size();) {
        size_t j = i;
        while (j < he.size() && he[j].key == he[i].key) ++j;
        if (j - i == 2) {
            E.ev.push_back(he[i].key / nv); E.ev.push_back(he[i].key % nv);
            E.etri.push_back(he[i].t); E.etri.push_back(he[i + 1].t);
            E.efree.push_back(he[i].w); E.efree.push_back(he[i + 1].w);
        }
        i = j;
    }
    if (E.etri.empty()) return fail(HM_ERR_ARG, "mesh has no interior edge");
    return HM_OK;
}

} // namespace

void launch_rhs_plane_wave(hm_matrix h, const double *d_k, const double *d_p, int nrhs, float2 *b, int64_t ldb,
                           cudaStream_t s)
{
    const int64_t total = h->N * nrhs;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    k_rhs_plane_wave<<<grid, 256, 0, s>>>(h->d_qpd, h->d_rhs_w, h->rhs_nq, h->d_vtx, h->d_ucell, h->d_ufree,
                                          h->d_ucoef, h->N, h->wavenumber, d_k, d_p, nrhs, b, ldb);
}

hm_status count_unknowns(const hm_mesh *mesh, int64_t *n)
{
    if (!mesh || !n) return fail(HM_ERR_ARG, "null argument");
    if (mesh->basis == HM_RWG) {
        RwgEdges E;
        hm_status st = rwg_edges(mesh, E);
        if (st != HM_OK) return st;
        *n = (int64_t)E.etri.size() / 2;
        return HM_OK;
    }
    if (mesh->basis == HM_SWG) {
        if (mesh->n_vert < 4 || mesh->n_cell < 1 || !mesh->xyz || !mesh->cells) return fail(HM_ERR_ARG, "empty mesh");
        std::vector<int32_t> fv, ft, ff;
        hm_status st = swg_faces(mesh->n_vert, mesh->n_cell, mesh->cells, fv, ft, ff);
        if (st != HM_OK) return st;
        *n = (int64_t)fv.size() / 3;
        return HM_OK;
    }
    return fail(HM_ERR_ARG, "unknown basis");
}

hm_status build_from_mesh(const hm_mesh *mesh, const hm_build_opts *o, cudaStream_t s, hm_matrix *out)
{
    if (o->leaf_size < 1 || o->leaf_size > factor_max_leaf())
        return fail(HM_ERR_ARG, "leaf_size must be in [1, " + std::to_string(factor_max_leaf()) + "]");
    if (o->arity != 2 && o->arity != 4 && o->arity != 8) return fail(HM_ERR_ARG, "arity must be 2, 4 or 8");
    if (!(o->adm > 0) || !(o->aca_tol > 0) || o->aca_tol >= 1) return fail(HM_ERR_ARG, "bad adm or aca_tol");
    if (!(mesh->wavelength > 0)) return fail(HM_ERR_ARG, "wavelength must be > 0");
    if (mesh->basis == HM_SWG) return build_from_tets(mesh, o, s, out);
    if (mesh->basis != HM_RWG) return fail(HM_ERR_ARG, "unknown basis");
    RwgEdges E;
    hm_status st = rwg_edges(mesh, E);
    if (st != HM_OK) return st;
    const int64_t nv = mesh->n_vert, nt = mesh->n_cell;
    const int64_t N = (int64_t)E.etri.size() / 2;
    BasisData B;
    B.N = N;
    std::vector<double> elen(N);
    for (int64_t i = 0; i < N; ++i) {
        const int64_t a = E.ev[2 * i], b = E.ev[2 * i + 1];
        const double *pa = mesh->xyz + 3 * a, *pb = mesh->xyz + 3 * b;
        const double dx = pa[0] - pb[0], dy = pa[1] - pb[1], dz = pa[2] - pb[2];
        elen[i] = std::sqrt(dx * dx + dy * dy + dz * dz);
        for (int d = 0; d < 3; ++d) B.cen.push_back(0.5 * (pa[d] + pb[d]));
        const int64_t vv[4] = {a, b, E.efree[2 * i], E.efree[2 * i + 1]};
        for (int d = 0; d < 3; ++d) {
            double lo = INFINITY, hi = -INFINITY;
            for (int q = 0; q < 4; ++q) {
                lo = std::min(lo, mesh->xyz[3 * vv[q] + d]);
                hi = std::max(hi, mesh->xyz[3 * vv[q] + d]);
            }
            B.blo.push_back(lo);
            B.bhi.push_back(hi);
        }
    }
    // ---- geometry on the device
    std::vector<double> area(nt), tcen(3 * nt), hmax(nt), nrm(3 * nt), qpd(3 * NQ * nt);
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
    const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
    const double bary[NQ][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {a1, a1, b1}, {a1, b1, a1}, {b1, a1, a1},
                                {a2, a2, b2}, {a2, b2, a2}, {b2, a2, a2}};
    const double qw[NQ] = {9.0 / 40.0, (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0,
                           (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0};
    for (int64_t t = 0; t < nt; ++t) {
        const double *p0 = mesh->xyz + 3 * mesh->cells[3 * t], *p1 = mesh->xyz + 3 * mesh->cells[3 * t + 1],
                     *p2 = mesh->xyz + 3 * mesh->cells[3 * t + 2];
        double e1[3], e2[3], e3[3], n[3];
        for (int d = 0; d < 3; ++d) { e1[d] = p1[d] - p0[d]; e2[d] = p2[d] - p0[d]; e3[d] = p2[d] - p1[d]; }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        area[t] = 0.5 * nn;
        for (int d = 0; d < 3; ++d) {
            nrm[3 * t + d] = n[d] / nn;
            tcen[3 * t + d] = (p0[d] + p1[d] + p2[d]) / 3.0;
        }
        const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        const double l2 = std::sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
        const double l3 = std::sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
        double hm_ = l1;
        if (l2 > hm_) hm_ = l2;
        if (l3 > hm_) hm_ = l3;
        hmax[t] = hm_;
        for (int q = 0; q < NQ; ++q)
            for (int d = 0; d < 3; ++d)
                qpd[(t * NQ + q) * 3 + d] = bary[q][0] * p0[d] + bary[q][1] * p1[d] + bary[q][2] * p2[d];
    }
    HM_CUDA(cudaMemcpyToSymbol(c_qw, qw, sizeof(qw)));
    TmpBuffers tmp;
    Geo g{};
    std::vector<double> vtx(mesh->xyz, mesh->xyz + 3 * nv);
    std::vector<int32_t> trv(mesh->cells, mesh->cells + 3 * nt);
    double *d_vtx, *d_cen, *d_hmax, *d_area, *d_nrm, *d_qpd, *d_elen;
    int32_t *d_tri, *d_etri, *d_efree;
    if ((st = tmp.up(&d_vtx, vtx, s)) || (st = tmp.up(&d_tri, trv, s)) || (st = tmp.up(&d_cen, tcen, s)) ||
        (st = tmp.up(&d_hmax, hmax, s)) || (st = tmp.up(&d_area, area, s)) || (st = tmp.up(&d_nrm, nrm, s)) ||
        (st = tmp.up(&d_qpd, qpd, s)) || (st = tmp.up(&d_etri, E.etri, s)) || (st = tmp.up(&d_efree, E.efree, s)) ||
        (st = tmp.up(&d_elen, elen, s)))
        return st;
    g.vtx = d_vtx; g.tri = d_tri; g.cen = d_cen; g.hmax = d_hmax; g.area = d_area; g.nrm = d_nrm; g.qpd = d_qpd;
    g.etri = d_etri; g.efree = d_efree; g.elen = d_elen;
    g.k = 2.0 * 3.14159265358979323846 / mesh->wavelength;
    g.eta = 376.730313461770655;

    B.nq = NQ;
    B.qw.assign(qw, qw + NQ);
    B.qpd = qpd;
    B.vtx = vtx;
    B.ucell = E.etri;
    B.ufree = E.efree;
    B.ucoef.resize(2 * N);
    for (int64_t i = 0; i < N; ++i) {
        B.ucoef[2 * i] = 0.5 * elen[i];
        B.ucoef[2 * i + 1] = -0.5 * elen[i];
    }
    st = assemble(B, g, o, tmp, s, out);
    if (st == HM_OK) (*out)->basis = HM_RWG;
    return st;
}

} // namespace hm
