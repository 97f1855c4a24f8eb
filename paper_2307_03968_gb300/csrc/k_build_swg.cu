// GPU construction of the V-EFIE H-Matrix of an inhomogeneous dielectric body
// from a tetrahedral mesh (arxiv 2307.03968 §II eq. 4, SWG basis [21]).
//
// Unknowns: one SWG function per face, D = eps0 sum_n x_n f_n; on T+
// f = +(a/3V)(r - v), on T- f = -(a/3V)(r - v), v the vertex opposite the
// face; boundary faces carry the T+ half only.  Contrast kappa = 1 - 1/eps_r
// per tetrahedron.  Eq. 4 (E_inc = D/eps + jwA + grad phi, polarisation current
// J = jw kappa D) tested with kappa f_m gives the complex-symmetric entries
//   Z_mn = Int (kappa/eps_r) f_m . f_n dV - k^2 Int Int kappa f_m . kappa' f_n' G
//          + Int Int q_m q_n' G,
// q the charge of kappa f: -kappa s a / V inside each tetrahedron (s = +-1 on
// T+/T-) and kappa(T+) - kappa(T-) on the function's own face (kappa(T+) on a
// boundary face).  The symmetric form is what makes the half storage of §III
// apply to the volume equation.
//
// Quadrature: 4-point degree-2 rule on tetrahedra, 7-point degree-5 rule on
// triangles.  Element pairs whose centroids are closer than 2 x the larger
// maximum edge length get the 1/R part of G analytically over the inner
// element: over a triangle from the edge form of the potential integrals
// (Wilton et al. 1984, Graglia 1993), over a tetrahedron by the divergence
// theorem, Int_T 1/R dV' = 1/2 sum_f ((p_f - r) . n_f) Int_f 1/R dS' and
// Int_T (r' - r)/R dV' = sum_f n_f Int_f R dS' with outward face normals n_f.
// Coordinates are taken relative to a vertex of the column face.  The near
// blocks (complex64) take the quadrature in FP32 but the analytic singular
// terms in FP64: the four tetrahedron pairs of one function pair cancel like a
// dipole-dipole interaction, which turns the ~1e-6 FP32 error of the edge
// formulas two or three element sizes away into ~1e-4 of the entry.  The leaf
// self blocks are filled entirely in FP64.
#include "k_assemble.cuh"

namespace hm {
namespace {

constexpr int NQT = 4;    // tetrahedron rule: barycentric (a,b,b,b) and permutations, weights 1/4
constexpr int NQF = 7;    // triangle rule (degree 5)
constexpr double EXTRACT_FACTOR = 2.0;
constexpr double INV4PI = 0.25 / 3.14159265358979323846;

__constant__ double c_fw[NQF];

struct VGeo {
    const double *vtx;      // nv x 3
    const int32_t *tet;     // nt x 4
    const double *tqp;      // nt x NQT x 3
    const double *tcen;     // nt x 3
    const double *thmax;    // nt
    const double *tvol;     // nt
    const double *kappa;    // nt
    const double *epsr;     // nt
    const int32_t *fv;      // nf x 3 (ascending)
    const int32_t *ftet;    // nf x 2 (T+, T- or -1)
    const int32_t *ffree;   // nf x 2
    const double *fqp;      // nf x NQF x 3
    const double *fcen;     // nf x 3
    const double *fhmax;    // nf
    const double *farea;    // nf
    const double *fqs;      // nf surface charge kappa(T+) - kappa(T-)
    const int32_t *perm;    // tree position -> original face index
    double k;
    template <class R> __device__ CX<R> entry(int m, int n) const;
};

// Singular-extraction predicate in FP64 without contractions (the same decision
// as any IEEE FP64 evaluation of |c_a - c_b|^2 < (2 max(h_a, h_b))^2).
__device__ __forceinline__ bool near_pair(const double *ca, double ha, const double *cb, double hb)
{
    const double dx = __dsub_rn(ca[0], cb[0]);
    const double dy = __dsub_rn(ca[1], cb[1]);
    const double dz = __dsub_rn(ca[2], cb[2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double h = ha > hb ? ha : hb;
    const double lim = __dmul_rn(EXTRACT_FACTOR, h);
    return d2 < __dmul_rn(lim, lim);
}

template <class R> __device__ __forceinline__ void loc(const double *p, const double *o, R out[3])
{
    out[0] = (R)(p[0] - o[0]);
    out[1] = (R)(p[1] - o[1]);
    out[2] = (R)(p[2] - o[2]);
}

template <class R> __device__ __forceinline__ R dot(const R a[3], const R b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// G (extract = false) or its smooth part G - 1/(4 pi R) (extract = true)
template <class R> __device__ __forceinline__ CX<R> green(R k, R Rr, bool extract)
{
    const R inv4pi = (R)(0.25 / 3.14159265358979323846);
    if (extract) {
        if (Rr < (R)1e-12) return CX<R>{0, -k * inv4pi};
        const R sh = sinR((R)0.5 * k * Rr);
        return CX<R>{-(R)2 * sh * sh * inv4pi / Rr, -sinR(k * Rr) * inv4pi / Rr};
    }
    R s, c;
    sincosR(k * Rr, &s, &c);
    return CX<R>{c * inv4pi / Rr, -s * inv4pi / Rr};
}

// Int_f 1/R dS' (s0) and Int_f R dS' (sR) over the flat triangle P at r, from the
// edge quantities of the potential integrals (Graglia 1993): per edge the
// signed in-plane distance t, the end coordinates l-, l+ and distances R-, R+;
// sR follows from div_s((rho' - rho) R) = 3R - d^2/R.
template <class R> __device__ void tri_s0_sR(const R P[3][3], const R r[3], R &s0, R &sR)
{
    const R e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    const R e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    R n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const R nn = sqrtR(dot(n, n));
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    const R rp[3] = {r[0] - P[0][0], r[1] - P[0][1], r[2] - P[0][2]};
    const R dd = dot(n, rp);
    const R ad = absR(dd);
    const R rho[3] = {r[0] - dd * n[0], r[1] - dd * n[1], r[2] - dd * n[2]};
    R acc0 = 0, edgeR = 0;
    for (int e = 0; e < 3; ++e) {
        const R *a = P[e], *b = P[(e + 1) % 3];
        const R lv[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const R ll = sqrtR(dot(lv, lv));
        const R lh[3] = {lv[0] / ll, lv[1] / ll, lv[2] / ll};
        const R uh[3] = {lh[1] * n[2] - lh[2] * n[1], lh[2] * n[0] - lh[0] * n[2], lh[0] * n[1] - lh[1] * n[0]};
        const R am[3] = {a[0] - rho[0], a[1] - rho[1], a[2] - rho[2]};
        const R bm[3] = {b[0] - rho[0], b[1] - rho[1], b[2] - rho[2]};
        const R lp = dot(bm, lh), lm = dot(am, lh), t = dot(am, uh);
        const R R02 = t * t + dd * dd;
        const R Rp = sqrtR(R02 + lp * lp), Rm = sqrtR(R02 + lm * lm);
        R f = 0;
        if (R02 > 0) {
            f = (lm < 0 && lp < 0) ? logR((Rm - lm) / (Rp - lp)) : logR((Rp + lp) / (Rm + lm));
            R term = t * f;
            if (ad > 0) term -= ad * (atanR(t * lp / (R02 + ad * Rp)) - atanR(t * lm / (R02 + ad * Rm)));
            acc0 += term;
        }
        const R gg = (R)0.5 * ((R02 > 0 ? R02 * f : (R)0) + lp * Rp - lm * Rm);
        edgeR += t * gg;
    }
    s0 = acc0;
    sR = (dd * dd * acc0 + edgeR) / (R)3;
}

template <class R> __device__ void face_local(const VGeo &g, int f, const double *o, R P[3][3])
{
    for (int a = 0; a < 3; ++a) loc<R>(g.vtx + 3 * g.fv[3 * f + a], o, P[a]);
}

// Int_T 1/R dV' (s0v) and Int_T (r' - r)/R dV' (s1v) for tetrahedron t at r
template <class R> __device__ void tet_integrals(const VGeo &g, int t, const double *o, const R r[3], R &s0v, R s1v[3])
{
    R P[4][3];
    for (int a = 0; a < 4; ++a) loc<R>(g.vtx + 3 * g.tet[4 * t + a], o, P[a]);
    s0v = 0;
    s1v[0] = s1v[1] = s1v[2] = 0;
    for (int op = 0; op < 4; ++op) {
        R F[3][3];
        int q = 0;
        for (int a = 0; a < 4; ++a)
            if (a != op) {
                F[q][0] = P[a][0]; F[q][1] = P[a][1]; F[q][2] = P[a][2];
                ++q;
            }
        const R e1[3] = {F[1][0] - F[0][0], F[1][1] - F[0][1], F[1][2] - F[0][2]};
        const R e2[3] = {F[2][0] - F[0][0], F[2][1] - F[0][1], F[2][2] - F[0][2]};
        R n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const R nn = sqrtR(dot(n, n));
        n[0] /= nn; n[1] /= nn; n[2] /= nn;
        const R po[3] = {P[op][0] - F[0][0], P[op][1] - F[0][1], P[op][2] - F[0][2]};
        if (dot(n, po) > 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }   // outward
        R s0, sR;
        tri_s0_sR<R>(F, r, s0, sR);
        const R pr[3] = {F[0][0] - r[0], F[0][1] - r[1], F[0][2] - r[2]};
        s0v += (R)0.5 * dot(pr, n) * s0;
        s1v[0] += n[0] * sR;
        s1v[1] += n[1] * sR;
        s1v[2] += n[2] * sR;
    }
}

// I = Int_T Int_T' (r - vm).(r' - vn) G,  J = Int_T Int_T' G  (T outer, T' inner)
template <class R>
__device__ void volvol(const VGeo &g, int t, int vmi, int tp, int vni, const double *o, CX<R> &I, CX<R> &J)
{
    const R k = (R)g.k;
    const bool ex = near_pair(g.tcen + 3 * t, g.thmax[t], g.tcen + 3 * tp, g.thmax[tp]);
    R vm[3], vn[3], qj[NQT][3];
    loc<R>(g.vtx + 3 * vmi, o, vm);
    loc<R>(g.vtx + 3 * vni, o, vn);
    for (int j = 0; j < NQT; ++j) loc<R>(g.tqp + ((int64_t)tp * NQT + j) * 3, o, qj[j]);
    const R Vt = (R)g.tvol[t], Vtp = (R)g.tvol[tp];
    I = CX<R>{0, 0};
    J = CX<R>{0, 0};
    for (int i = 0; i < NQT; ++i) {
        R ri[3];
        loc<R>(g.tqp + ((int64_t)t * NQT + i) * 3, o, ri);
        const R a[3] = {ri[0] - vm[0], ri[1] - vm[1], ri[2] - vm[2]};
        CX<R> Ii{0, 0}, Ji{0, 0};
        for (int j = 0; j < NQT; ++j) {
            const R bj[3] = {qj[j][0] - vn[0], qj[j][1] - vn[1], qj[j][2] - vn[2]};
            const R dr[3] = {ri[0] - qj[j][0], ri[1] - qj[j][1], ri[2] - qj[j][2]};
            const CX<R> G = green<R>(k, sqrtR(dot(dr, dr)), ex);
            const R w = (R)0.25 * dot(a, bj);
            Ii.re += w * G.re; Ii.im += w * G.im;
            Ji.re += (R)0.25 * G.re; Ji.im += (R)0.25 * G.im;
        }
        Ii.re *= Vtp; Ii.im *= Vtp; Ji.re *= Vtp; Ji.im *= Vtp;
        if (ex) {   // analytic 1/R part in FP64 (see the note on precision above)
            double rd[3], vmd[3], vnd[3], s0v, s1v[3];
            loc<double>(g.tqp + ((int64_t)t * NQT + i) * 3, o, rd);
            loc<double>(g.vtx + 3 * vmi, o, vmd);
            loc<double>(g.vtx + 3 * vni, o, vnd);
            tet_integrals<double>(g, tp, o, rd, s0v, s1v);
            const double ad[3] = {rd[0] - vmd[0], rd[1] - vmd[1], rd[2] - vmd[2]};
            const double v1[3] = {s1v[0] + (rd[0] - vnd[0]) * s0v, s1v[1] + (rd[1] - vnd[1]) * s0v,
                                  s1v[2] + (rd[2] - vnd[2]) * s0v};
            Ii.re += (R)(dot(ad, v1) * INV4PI);
            Ji.re += (R)(s0v * INV4PI);
        }
        I.re += (R)0.25 * Ii.re; I.im += (R)0.25 * Ii.im;
        J.re += (R)0.25 * Ji.re; J.im += (R)0.25 * Ji.im;
    }
    I.re *= Vt; I.im *= Vt; J.re *= Vt; J.im *= Vt;
}

// Int_T Int_f G dS' dV  (tetrahedron t outer, face f inner)
template <class R> __device__ CX<R> volface(const VGeo &g, int t, int f, const double *o)
{
    const R k = (R)g.k;
    const bool ex = near_pair(g.tcen + 3 * t, g.thmax[t], g.fcen + 3 * f, g.fhmax[f]);
    double P[3][3];
    if (ex) face_local<double>(g, f, o, P);
    CX<R> K{0, 0};
    for (int i = 0; i < NQT; ++i) {
        R ri[3];
        loc<R>(g.tqp + ((int64_t)t * NQT + i) * 3, o, ri);
        CX<R> Ki{0, 0};
        for (int j = 0; j < NQF; ++j) {
            R rj[3];
            loc<R>(g.fqp + ((int64_t)f * NQF + j) * 3, o, rj);
            const R dr[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
            const CX<R> G = green<R>(k, sqrtR(dot(dr, dr)), ex);
            const R w = (R)c_fw[j];
            Ki.re += w * G.re; Ki.im += w * G.im;
        }
        const R A = (R)g.farea[f];
        Ki.re *= A; Ki.im *= A;
        if (ex) {
            double rd[3], s0, sR;
            loc<double>(g.tqp + ((int64_t)t * NQT + i) * 3, o, rd);
            tri_s0_sR<double>(P, rd, s0, sR);
            Ki.re += (R)(s0 * INV4PI);
        }
        K.re += (R)0.25 * Ki.re; K.im += (R)0.25 * Ki.im;
    }
    const R Vt = (R)g.tvol[t];
    K.re *= Vt; K.im *= Vt;
    return K;
}

// Int_f Int_f' G dS' dS  (f outer, f' inner)
template <class R> __device__ CX<R> faceface(const VGeo &g, int f, int fp, const double *o)
{
    const R k = (R)g.k;
    const bool ex = near_pair(g.fcen + 3 * f, g.fhmax[f], g.fcen + 3 * fp, g.fhmax[fp]);
    double P[3][3];
    if (ex) face_local<double>(g, fp, o, P);
    CX<R> L{0, 0};
    for (int i = 0; i < NQF; ++i) {
        R ri[3];
        loc<R>(g.fqp + ((int64_t)f * NQF + i) * 3, o, ri);
        CX<R> Li{0, 0};
        for (int j = 0; j < NQF; ++j) {
            R rj[3];
            loc<R>(g.fqp + ((int64_t)fp * NQF + j) * 3, o, rj);
            const R dr[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
            const CX<R> G = green<R>(k, sqrtR(dot(dr, dr)), ex);
            const R w = (R)c_fw[j];
            Li.re += w * G.re; Li.im += w * G.im;
        }
        const R A = (R)g.farea[fp];
        Li.re *= A; Li.im *= A;
        if (ex) {
            double rd[3], s0, sR;
            loc<double>(g.fqp + ((int64_t)f * NQF + i) * 3, o, rd);
            tri_s0_sR<double>(P, rd, s0, sR);
            Li.re += (R)(s0 * INV4PI);
        }
        const R w = (R)c_fw[i];
        L.re += w * Li.re; L.im += w * Li.im;
    }
    const R A = (R)g.farea[f];
    L.re *= A; L.im *= A;
    return L;
}

template <class R> __device__ CX<R> VGeo::entry(int m, int n) const
{
    const VGeo &g = *this;
    const double *o = g.vtx + 3 * g.fv[3 * n];
    const double k2 = g.k * g.k;
    const double qs_m = g.fqs[m], qs_n = g.fqs[n];
    CX<R> z{0, 0};
    for (int p = 0; p < 2; ++p) {
        const int t = g.ftet[2 * m + p];
        if (t < 0) continue;
        const double s = p == 0 ? 1.0 : -1.0;
        const int vm = g.ffree[2 * m + p];
        const double cm = s * g.farea[m] / (3.0 * g.tvol[t]);
        const double qm = -g.kappa[t] * s * g.farea[m] / g.tvol[t];
        for (int q = 0; q < 2; ++q) {
            const int tp = g.ftet[2 * n + q];
            if (tp < 0) continue;
            const double sp = q == 0 ? 1.0 : -1.0;
            const int vn = g.ffree[2 * n + q];
            const double cn = sp * g.farea[n] / (3.0 * g.tvol[tp]);
            const double qn = -g.kappa[tp] * sp * g.farea[n] / g.tvol[tp];
            if (t == tp) {   // Int (kappa/eps_r) f_m . f_n dV: degree 2, exact with the 4-point rule
                R vmr[3], vnr[3];
                loc<R>(g.vtx + 3 * vm, o, vmr);
                loc<R>(g.vtx + 3 * vn, o, vnr);
                R acc = 0;
                for (int i = 0; i < NQT; ++i) {
                    R ri[3];
                    loc<R>(g.tqp + ((int64_t)t * NQT + i) * 3, o, ri);
                    const R a[3] = {ri[0] - vmr[0], ri[1] - vmr[1], ri[2] - vmr[2]};
                    const R b[3] = {ri[0] - vnr[0], ri[1] - vnr[1], ri[2] - vnr[2]};
                    acc += (R)0.25 * dot(a, b);
                }
                z.re += (R)(g.kappa[t] / g.epsr[t] * cm * cn * g.tvol[t]) * acc;
            }
            CX<R> I, J;
            volvol<R>(g, t, vm, tp, vn, o, I, J);
            const R ca = (R)(-k2 * g.kappa[t] * g.kappa[tp] * cm * cn), cb = (R)(qm * qn);
            z.re += ca * I.re + cb * J.re;
            z.im += ca * I.im + cb * J.im;
        }
        if (qs_n != 0.0) {
            const CX<R> K = volface<R>(g, t, n, o);
            const R c = (R)(qm * qs_n);
            z.re += c * K.re;
            z.im += c * K.im;
        }
    }
    if (qs_m != 0.0) {
        for (int q = 0; q < 2; ++q) {
            const int tp = g.ftet[2 * n + q];
            if (tp < 0) continue;
            const double sp = q == 0 ? 1.0 : -1.0;
            const double qn = -g.kappa[tp] * sp * g.farea[n] / g.tvol[tp];
            const CX<R> K = volface<R>(g, tp, m, o);   // = Int_{face m} Int_{tp} G
            const R c = (R)(qs_m * qn);
            z.re += c * K.re;
            z.im += c * K.im;
        }
        if (qs_n != 0.0) {
            const CX<R> L = faceface<R>(g, m, n, o);
            const R c = (R)(qs_m * qs_n);
            z.re += c * L.re;
            z.im += c * L.im;
        }
    }
    return z;
}

static double norm3(const double *d) { return std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]); }

static double max_edge(const double *const *p, int np)
{
    double h = 0.0;
    for (int i = 0; i < np; ++i)
        for (int j = i + 1; j < np; ++j) {
            const double d[3] = {p[i][0] - p[j][0], p[i][1] - p[j][1], p[i][2] - p[j][2]};
            const double l = norm3(d);
            if (l > h) h = l;
        }
    return h;
}

} // namespace

hm_status swg_faces(int64_t nv, int64_t nt, const int32_t *tet, std::vector<int32_t> &fv, std::vector<int32_t> &ftet,
                    std::vector<int32_t> &ffree)
{
    struct HF { std::array<int32_t, 3> key; int32_t t, w; };
    std::vector<HF> hf;
    hf.reserve(4 * nt);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *v = tet + 4 * t;
        for (int a = 0; a < 4; ++a) {
            if (v[a] < 0 || v[a] >= nv) return fail(HM_ERR_ARG, "tetrahedron vertex id out of range");
            for (int b = a + 1; b < 4; ++b)
                if (v[a] == v[b]) return fail(HM_ERR_ARG, "tetrahedron with a repeated vertex");
        }
        for (int op = 0; op < 4; ++op) {
            std::array<int32_t, 3> k{};
            int q = 0;
            for (int a = 0; a < 4; ++a)
                if (a != op) k[q++] = v[a];
            std::sort(k.begin(), k.end());
            hf.push_back({k, (int32_t)t, v[op]});
        }
    }
    std::sort(hf.begin(), hf.end(), [](const HF &x, const HF &y) { return x.key < y.key || (x.key == y.key && x.t < y.t); });
    fv.clear(); ftet.clear(); ffree.clear();
    for (size_t i = 0; i < hf.size();) {
        size_t j = i;
        while (j < hf.size() && hf[j].key == hf[i].key) ++j;
        if (j - i > 2) return fail(HM_ERR_ARG, "a face is shared by more than two tetrahedra");
        fv.insert(fv.end(), hf[i].key.begin(), hf[i].key.end());
        ftet.push_back(hf[i].t);
        ffree.push_back(hf[i].w);
        ftet.push_back(j - i == 2 ? hf[i + 1].t : -1);
        ffree.push_back(j - i == 2 ? hf[i + 1].w : -1);
        i = j;
    }
    return HM_OK;
}

hm_status build_from_tets(const hm_mesh *mesh, const hm_build_opts *o, cudaStream_t s, hm_matrix *out)
{
    const int64_t nv = mesh->n_vert, nt = mesh->n_cell;
    if (nv < 4 || nt < 1 || !mesh->xyz || !mesh->cells) return fail(HM_ERR_ARG, "empty mesh");
    if (!mesh->eps_r) return fail(HM_ERR_ARG, "eps_r is required for an SWG mesh");
    for (int64_t t = 0; t < nt; ++t)
        if (!(mesh->eps_r[t] > 0) || !std::isfinite(mesh->eps_r[t])) return fail(HM_ERR_ARG, "eps_r must be finite and > 0");
    std::vector<int32_t> fv, ftet, ffree;
    hm_status st = swg_faces(nv, nt, mesh->cells, fv, ftet, ffree);
    if (st != HM_OK) return st;
    const int64_t N = (int64_t)fv.size() / 3;
    const double *X = mesh->xyz;

    // ---- tetrahedra
    const double ta = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, tb = (5.0 - std::sqrt(5.0)) / 20.0;
    std::vector<double> tqp(3 * NQT * nt), tcen(3 * nt), thmax(nt), tvol(nt), kappa(nt), epsr(mesh->eps_r, mesh->eps_r + nt);
    for (int64_t t = 0; t < nt; ++t) {
        const double *p[4];
        for (int a = 0; a < 4; ++a) p[a] = X + 3 * mesh->cells[4 * t + a];
        const double e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
        const double e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
        const double e3[3] = {p[3][0] - p[0][0], p[3][1] - p[0][1], p[3][2] - p[0][2]};
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        tvol[t] = std::fabs(cr[0] * e3[0] + cr[1] * e3[1] + cr[2] * e3[2]) / 6.0;
        if (!(tvol[t] > 0)) return fail(HM_ERR_ARG, "degenerate tetrahedron (zero volume)");
        for (int d = 0; d < 3; ++d) tcen[3 * t + d] = (p[0][d] + p[1][d] + p[2][d] + p[3][d]) / 4.0;
        thmax[t] = max_edge(p, 4);
        kappa[t] = 1.0 - 1.0 / epsr[t];
        for (int q = 0; q < NQT; ++q)
            for (int d = 0; d < 3; ++d) {
                double acc = 0.0;
                for (int a = 0; a < 4; ++a) acc = acc + (q == a ? ta : tb) * p[a][d];
                tqp[(t * NQT + q) * 3 + d] = acc;
            }
    }
    // ---- faces
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
    const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
    const double bary[NQF][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {a1, a1, b1}, {a1, b1, a1}, {b1, a1, a1},
                                 {a2, a2, b2}, {a2, b2, a2}, {b2, a2, a2}};
    const double fw[NQF] = {9.0 / 40.0, (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0,
                            (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0};
    std::vector<double> fqp(3 * NQF * N), fcen(3 * N), fhmax(N), farea(N), fqs(N);
    BasisData B;
    B.N = N;
    for (int64_t f = 0; f < N; ++f) {
        const double *p[3];
        for (int a = 0; a < 3; ++a) p[a] = X + 3 * fv[3 * f + a];
        const double e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
        const double e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        farea[f] = 0.5 * norm3(cr);
        for (int d = 0; d < 3; ++d) fcen[3 * f + d] = (p[0][d] + p[1][d] + p[2][d]) / 3.0;
        fhmax[f] = max_edge(p, 3);
        for (int q = 0; q < NQF; ++q)
            for (int d = 0; d < 3; ++d)
                fqp[(f * NQF + q) * 3 + d] = bary[q][0] * p[0][d] + bary[q][1] * p[1][d] + bary[q][2] * p[2][d];
        const int tp = ftet[2 * f], tm = ftet[2 * f + 1];
        fqs[f] = kappa[tp] - (tm >= 0 ? kappa[tm] : 0.0);
        // tree: face centroid; support box: the vertices of T+ and T-
        for (int d = 0; d < 3; ++d) B.cen.push_back(fcen[3 * f + d]);
        const double *pp[5] = {p[0], p[1], p[2], X + 3 * ffree[2 * f], X + 3 * (tm >= 0 ? ffree[2 * f + 1] : ffree[2 * f])};
        for (int d = 0; d < 3; ++d) {
            double lo = INFINITY, hi = -INFINITY;
            for (int q = 0; q < 5; ++q) {
                lo = std::min(lo, pp[q][d]);
                hi = std::max(hi, pp[q][d]);
            }
            B.blo.push_back(lo);
            B.bhi.push_back(hi);
        }
    }
    HM_CUDA(cudaMemcpyToSymbol(c_fw, fw, sizeof(fw)));
    TmpBuffers tmp;
    std::vector<double> vtx(X, X + 3 * nv);
    std::vector<int32_t> tetv(mesh->cells, mesh->cells + 4 * nt);
    VGeo g{};
    double *d_vtx, *d_tqp, *d_tcen, *d_thmax, *d_tvol, *d_kappa, *d_epsr, *d_fqp, *d_fcen, *d_fhmax, *d_farea, *d_fqs;
    int32_t *d_tet, *d_fv, *d_ftet, *d_ffree;
    if ((st = tmp.up(&d_vtx, vtx, s)) || (st = tmp.up(&d_tet, tetv, s)) || (st = tmp.up(&d_tqp, tqp, s)) ||
        (st = tmp.up(&d_tcen, tcen, s)) || (st = tmp.up(&d_thmax, thmax, s)) || (st = tmp.up(&d_tvol, tvol, s)) ||
        (st = tmp.up(&d_kappa, kappa, s)) || (st = tmp.up(&d_epsr, epsr, s)) || (st = tmp.up(&d_fv, fv, s)) ||
        (st = tmp.up(&d_ftet, ftet, s)) || (st = tmp.up(&d_ffree, ffree, s)) || (st = tmp.up(&d_fqp, fqp, s)) ||
        (st = tmp.up(&d_fcen, fcen, s)) || (st = tmp.up(&d_fhmax, fhmax, s)) || (st = tmp.up(&d_farea, farea, s)) ||
        (st = tmp.up(&d_fqs, fqs, s)))
        return st;
    g.vtx = d_vtx; g.tet = d_tet; g.tqp = d_tqp; g.tcen = d_tcen; g.thmax = d_thmax; g.tvol = d_tvol;
    g.kappa = d_kappa; g.epsr = d_epsr; g.fv = d_fv; g.ftet = d_ftet; g.ffree = d_ffree; g.fqp = d_fqp;
    g.fcen = d_fcen; g.fhmax = d_fhmax; g.farea = d_farea; g.fqs = d_fqs;
    g.k = 2.0 * 3.14159265358979323846 / mesh->wavelength;

    // excitation: b_m = sum_s (s kappa_s a / 3) sum_q (1/4) (r_q - v_s) . p exp(-jk k . r_q)
    B.nq = NQT;
    B.qw.assign(NQT, 0.25);
    B.qpd = tqp;
    B.vtx = vtx;
    B.ucell = ftet;
    B.ufree = ffree;
    B.ucoef.resize(2 * N);
    for (int64_t f = 0; f < N; ++f)
        for (int p = 0; p < 2; ++p) {
            const int t = ftet[2 * f + p];
            B.ucoef[2 * f + p] = t < 0 ? 0.0 : (p == 0 ? 1.0 : -1.0) * kappa[t] * farea[f] / 3.0;
        }
    st = assemble(B, g, o, tmp, s, out);
    if (st == HM_OK) (*out)->basis = HM_SWG;
    return st;
}

} // namespace hm
