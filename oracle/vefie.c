/*
 * CPU oracle, complex128 — TEST INFRASTRUCTURE ONLY (see efie.c).
 *
 * Volume EFIE of an inhomogeneous dielectric body with SWG basis functions
 * (arxiv 2307.03968 §II, eq. 4, "SWG basis function for volume V-EFIE"; SWG =
 * Schaubert, Wilton & Glisson 1984).  Time convention e^{jwt}, G = e^{-jkR}/(4 pi R).
 *
 * Unknowns: D = eps0 sum_n x_n f_n (x in V/m), one SWG function per face of the
 * tetrahedral mesh: on T+ f = +(a/3V)(r - v), on T- f = -(a/3V)(r - v), v the
 * free vertex, a the face area; boundary faces carry the T+ half only.
 * Contrast kappa = 1 - 1/eps_r per tetrahedron; polarisation current
 * J = jw kappa D; charge of kappa f: volume -kappa div f inside each
 * tetrahedron, surface kappa(T+) - kappa(T-) on the function's face (kappa(T+)
 * on a boundary face).
 *
 * Eq. 4, E_inc = D/eps + jw A + grad phi, is tested with kappa f_m (which makes
 * the matrix complex symmetric, so the half storage of §III applies):
 *   Z_mn = Int (kappa/eps_r) f_m.f_n dV
 *        - k^2 Int Int kappa f_m . kappa' f_n' G dV' dV
 *        + Int Int q_m q_n' G                       (volume and surface charges)
 *   b_m  = Int kappa f_m . E_inc dV.
 *
 * Quadrature: 4-point degree-2 rule on tetrahedra, 7-point degree-5 rule on
 * triangles.  Element pairs whose centroids are closer than 2 x the larger
 * maximum edge length get the 1/R part of G analytically over the inner
 * element: over a triangle with the potential integrals of efie.c; over a
 * tetrahedron by the divergence theorem,
 *   Int_T 1/R dV'        = 1/2 sum_faces ((p_f - r).n_f) Int_f 1/R dS'
 *   Int_T (r'-r)/R dV'   = sum_faces n_f Int_f R dS'      (n_f outward).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zc;

void hmo_potential_integrals3(const double *p0, const double *p1, const double *p2, const double *r,
                              double *s0_out, double *s1v_out, double *sR_out);
typedef zc (*hmo_entry_fn)(const void *ctx, int m, int n);
int hmo_aca_generic(hmo_entry_fn entry, const void *c, const int32_t *rows, int m, const int32_t *cols, int n,
                    double tol, int kmax, zc *U, zc *V);
void hmo_aca_many_generic(hmo_entry_fn entry, const void *c, int nb, const int32_t *idx, const int64_t *roff,
                          const int32_t *m, const int64_t *coff, const int32_t *n, double tol, const int32_t *kmax,
                          const int64_t *uoff, const int64_t *voff, zc *U, zc *V, int32_t *rank);

#define NQT 4
#define NQF 7
#define EXTRACT_FACTOR 2.0

typedef struct {
    int nv, nt, nf;
    const double *xyz;
    const int32_t *tet;      /* nt x 4 */
    const double *epsr;      /* nt */
    const int32_t *ftet;     /* nf x 2: T+, T- (-1 on the boundary) */
    const int32_t *ffree;    /* nf x 2: free vertex in T+, in T- */
    const int32_t *fvert;    /* nf x 3 */
    double k;
    double *tvol, *tcen, *thmax, *tqp, *kappa;
    double *farea, *fcen, *fhmax, *fqp;
    double tw[NQT], fw[NQF];
} vmo_ctx;

static inline void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double norm3(const double *a) { return sqrt(dot3(a, a)); }

static double max_edge(const double *const *p, int np)
{
    double h = 0.0;
    for (int i = 0; i < np; ++i)
        for (int j = i + 1; j < np; ++j) {
            double d[3];
            sub3(p[i], p[j], d);
            if (norm3(d) > h) h = norm3(d);
        }
    return h;
}

vmo_ctx *vmo_ctx_new(int nv, const double *xyz, int nt, const int32_t *tet, const double *epsr, int nf,
                     const int32_t *ftet, const int32_t *ffree, const int32_t *fvert, double k)
{
    vmo_ctx *c = (vmo_ctx *)calloc(1, sizeof(vmo_ctx));
    c->nv = nv; c->nt = nt; c->nf = nf;
    c->xyz = xyz; c->tet = tet; c->epsr = epsr; c->ftet = ftet; c->ffree = ffree; c->fvert = fvert; c->k = k;
    c->tvol = malloc(sizeof(double) * nt);
    c->tcen = malloc(sizeof(double) * nt * 3);
    c->thmax = malloc(sizeof(double) * nt);
    c->tqp = malloc(sizeof(double) * nt * NQT * 3);
    c->kappa = malloc(sizeof(double) * nt);
    c->farea = malloc(sizeof(double) * nf);
    c->fcen = malloc(sizeof(double) * nf * 3);
    c->fhmax = malloc(sizeof(double) * nf);
    c->fqp = malloc(sizeof(double) * nf * NQF * 3);
    /* tetrahedron rule: barycentric (a, b, b, b) and permutations, weights 1/4 */
    const double ta = (5.0 + 3.0 * sqrt(5.0)) / 20.0, tb = (5.0 - sqrt(5.0)) / 20.0;
    double tbary[NQT][4];
    for (int q = 0; q < NQT; ++q)
        for (int v = 0; v < 4; ++v) tbary[q][v] = (q == v) ? ta : tb;
    for (int q = 0; q < NQT; ++q) c->tw[q] = 0.25;
    for (int t = 0; t < nt; ++t) {
        const double *p[4];
        for (int v = 0; v < 4; ++v) p[v] = xyz + 3 * tet[4 * t + v];
        double e1[3], e2[3], e3[3], cr[3];
        sub3(p[1], p[0], e1); sub3(p[2], p[0], e2); sub3(p[3], p[0], e3);
        cross3(e1, e2, cr);
        c->tvol[t] = fabs(dot3(cr, e3)) / 6.0;
        for (int d = 0; d < 3; ++d) c->tcen[3 * t + d] = (p[0][d] + p[1][d] + p[2][d] + p[3][d]) / 4.0;
        c->thmax[t] = max_edge(p, 4);
        c->kappa[t] = 1.0 - 1.0 / epsr[t];
        for (int q = 0; q < NQT; ++q)
            for (int d = 0; d < 3; ++d)
                c->tqp[(t * NQT + q) * 3 + d] = tbary[q][0] * p[0][d] + tbary[q][1] * p[1][d] +
                                               tbary[q][2] * p[2][d] + tbary[q][3] * p[3][d];
    }
    /* triangle rule (the same closed-form 7-point rule as efie.c) */
    const double s15 = sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
    const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    const double fbary[NQF][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {a1, a1, b1}, {a1, b1, a1}, {b1, a1, a1},
                                  {a2, a2, b2}, {a2, b2, a2}, {b2, a2, a2}};
    const double fw[NQF] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    memcpy(c->fw, fw, sizeof(fw));
    for (int f = 0; f < nf; ++f) {
        const double *p[3];
        for (int v = 0; v < 3; ++v) p[v] = xyz + 3 * fvert[3 * f + v];
        double e1[3], e2[3], cr[3];
        sub3(p[1], p[0], e1); sub3(p[2], p[0], e2);
        cross3(e1, e2, cr);
        c->farea[f] = 0.5 * norm3(cr);
        for (int d = 0; d < 3; ++d) c->fcen[3 * f + d] = (p[0][d] + p[1][d] + p[2][d]) / 3.0;
        c->fhmax[f] = max_edge(p, 3);
        for (int q = 0; q < NQF; ++q)
            for (int d = 0; d < 3; ++d)
                c->fqp[(f * NQF + q) * 3 + d] = fbary[q][0] * p[0][d] + fbary[q][1] * p[1][d] + fbary[q][2] * p[2][d];
    }
    return c;
}

void vmo_ctx_free(vmo_ctx *c)
{
    if (!c) return;
    free(c->tvol); free(c->tcen); free(c->thmax); free(c->tqp); free(c->kappa);
    free(c->farea); free(c->fcen); free(c->fhmax); free(c->fqp);
    free(c);
}

static int extract(const double *ca, double ha, const double *cb, double hb)
{
    double d[3];
    sub3(ca, cb, d);
    const double h = ha > hb ? ha : hb;
    return dot3(d, d) < (EXTRACT_FACTOR * h) * (EXTRACT_FACTOR * h);
}

/* G and its smooth remainder (G - 1/(4 pi R)) */
static zc green(double k, double R) { return cexp(-I * k * R) / (4.0 * M_PI * R); }
static zc green_smooth(double k, double R)
{
    if (R < 1e-14) return -I * k / (4.0 * M_PI);
    const double sh = sin(0.5 * k * R);
    return (-2.0 * sh * sh - I * sin(k * R)) / (4.0 * M_PI * R);
}

/* Int_T 1/R dV' and Int_T (r'-r)/R dV' for tetrahedron t at point r */
void vmo_volume_integrals(const vmo_ctx *c, int t, const double *r, double *s0v, double *s1v)
{
    const int32_t *tv = c->tet + 4 * t;
    *s0v = 0.0;
    s1v[0] = s1v[1] = s1v[2] = 0.0;
    for (int o = 0; o < 4; ++o) {   /* face opposite vertex o */
        const double *p[3];
        int q = 0;
        for (int v = 0; v < 4; ++v)
            if (v != o) p[q++] = c->xyz + 3 * tv[v];
        double e1[3], e2[3], nrm[3], po[3];
        sub3(p[1], p[0], e1); sub3(p[2], p[0], e2);
        cross3(e1, e2, nrm);
        const double nn = norm3(nrm);
        for (int d = 0; d < 3; ++d) nrm[d] /= nn;
        sub3(c->xyz + 3 * tv[o], p[0], po);
        if (dot3(nrm, po) > 0) for (int d = 0; d < 3; ++d) nrm[d] = -nrm[d];   /* outward */
        double s0, s1[3], sR, pr[3];
        hmo_potential_integrals3(p[0], p[1], p[2], r, &s0, s1, &sR);
        sub3(p[0], r, pr);
        *s0v += 0.5 * dot3(pr, nrm) * s0;
        for (int d = 0; d < 3; ++d) s1v[d] += nrm[d] * sR;
    }
}

/* I = Int_T Int_T' (r - vm).(r' - vn) G,  J = Int_T Int_T' G  (T outer, T' inner) */
static void volvol(const vmo_ctx *c, int t, const double *vm, int tp, const double *vn, zc *I_out, zc *J_out)
{
    const double k = c->k;
    const int ex = extract(c->tcen + 3 * t, c->thmax[t], c->tcen + 3 * tp, c->thmax[tp]);
    zc Ivv = 0.0, Jvv = 0.0;
    for (int i = 0; i < NQT; ++i) {
        const double *ri = c->tqp + (t * NQT + i) * 3;
        double a[3];
        sub3(ri, vm, a);
        zc Ii = 0.0, Ji = 0.0;
        for (int j = 0; j < NQT; ++j) {
            const double *rj = c->tqp + (tp * NQT + j) * 3;
            double bj[3], dr[3];
            sub3(rj, vn, bj);
            sub3(ri, rj, dr);
            const double R = norm3(dr);
            const zc g = ex ? green_smooth(k, R) : green(k, R);
            Ii += c->tw[j] * dot3(a, bj) * g;
            Ji += c->tw[j] * g;
        }
        Ii *= c->tvol[tp];
        Ji *= c->tvol[tp];
        if (ex) {
            double s0v, s1v[3], rv[3];
            vmo_volume_integrals(c, tp, ri, &s0v, s1v);
            sub3(ri, vn, rv);
            double v1[3] = {s1v[0] + rv[0] * s0v, s1v[1] + rv[1] * s0v, s1v[2] + rv[2] * s0v};
            Ii += dot3(a, v1) / (4.0 * M_PI);
            Ji += s0v / (4.0 * M_PI);
        }
        Ivv += c->tw[i] * Ii;
        Jvv += c->tw[i] * Ji;
    }
    *I_out = Ivv * c->tvol[t];
    *J_out = Jvv * c->tvol[t];
}

/* Int_T Int_f G dS' dV  (tetrahedron t outer, face f inner) */
static zc volface(const vmo_ctx *c, int t, int f)
{
    const double k = c->k;
    const int ex = extract(c->tcen + 3 * t, c->thmax[t], c->fcen + 3 * f, c->fhmax[f]);
    zc K = 0.0;
    for (int i = 0; i < NQT; ++i) {
        const double *ri = c->tqp + (t * NQT + i) * 3;
        zc Ki = 0.0;
        for (int j = 0; j < NQF; ++j) {
            const double *rj = c->fqp + (f * NQF + j) * 3;
            double dr[3];
            sub3(ri, rj, dr);
            const double R = norm3(dr);
            Ki += c->fw[j] * (ex ? green_smooth(k, R) : green(k, R));
        }
        Ki *= c->farea[f];
        if (ex) {
            const int32_t *fv = c->fvert + 3 * f;
            double s0, s1[3];
            hmo_potential_integrals3(c->xyz + 3 * fv[0], c->xyz + 3 * fv[1], c->xyz + 3 * fv[2], ri, &s0, s1, NULL);
            Ki += s0 / (4.0 * M_PI);
        }
        K += c->tw[i] * Ki;
    }
    return K * c->tvol[t];
}

/* Int_f Int_f' G dS' dS  (f outer, f' inner) */
static zc faceface(const vmo_ctx *c, int f, int fp)
{
    const double k = c->k;
    const int ex = extract(c->fcen + 3 * f, c->fhmax[f], c->fcen + 3 * fp, c->fhmax[fp]);
    zc L = 0.0;
    for (int i = 0; i < NQF; ++i) {
        const double *ri = c->fqp + (f * NQF + i) * 3;
        zc Li = 0.0;
        for (int j = 0; j < NQF; ++j) {
            const double *rj = c->fqp + (fp * NQF + j) * 3;
            double dr[3];
            sub3(ri, rj, dr);
            const double R = norm3(dr);
            Li += c->fw[j] * (ex ? green_smooth(k, R) : green(k, R));
        }
        Li *= c->farea[fp];
        if (ex) {
            const int32_t *fv = c->fvert + 3 * fp;
            double s0, s1[3];
            hmo_potential_integrals3(c->xyz + 3 * fv[0], c->xyz + 3 * fv[1], c->xyz + 3 * fv[2], ri, &s0, s1, NULL);
            Li += s0 / (4.0 * M_PI);
        }
        L += c->fw[i] * Li;
    }
    return L * c->farea[f];
}

/* surface charge of kappa f on its own face */
static double face_charge(const vmo_ctx *c, int m)
{
    const int tp = c->ftet[2 * m], tm = c->ftet[2 * m + 1];
    return c->kappa[tp] - (tm >= 0 ? c->kappa[tm] : 0.0);
}

zc vmo_entry(const vmo_ctx *c, int m, int n)
{
    const double k2 = c->k * c->k;
    const double qs_m = face_charge(c, m), qs_n = face_charge(c, n);
    zc z = 0.0;
    for (int p = 0; p < 2; ++p) {
        const int t = c->ftet[2 * m + p];
        if (t < 0) continue;
        const double s = p == 0 ? 1.0 : -1.0;
        const double *vm = c->xyz + 3 * c->ffree[2 * m + p];
        const double cm = s * c->farea[m] / (3.0 * c->tvol[t]);          /* f_m = cm (r - vm) on t */
        const double qm = -c->kappa[t] * s * c->farea[m] / c->tvol[t];   /* volume charge of kappa f_m */
        for (int q = 0; q < 2; ++q) {
            const int tp = c->ftet[2 * n + q];
            if (tp < 0) continue;
            const double sp = q == 0 ? 1.0 : -1.0;
            const double *vn = c->xyz + 3 * c->ffree[2 * n + q];
            const double cn = sp * c->farea[n] / (3.0 * c->tvol[tp]);
            const double qn = -c->kappa[tp] * sp * c->farea[n] / c->tvol[tp];
            if (t == tp) {   /* Int (kappa/eps_r) f_m.f_n dV, degree 2: exact with the 4-point rule */
                double acc = 0.0;
                for (int i = 0; i < NQT; ++i) {
                    const double *ri = c->tqp + (t * NQT + i) * 3;
                    double a[3], b[3];
                    sub3(ri, vm, a);
                    sub3(ri, vn, b);
                    acc += c->tw[i] * dot3(a, b);
                }
                z += c->kappa[t] / c->epsr[t] * cm * cn * acc * c->tvol[t];
            }
            zc Ivv, Jvv;
            volvol(c, t, vm, tp, vn, &Ivv, &Jvv);
            z += -k2 * c->kappa[t] * c->kappa[tp] * cm * cn * Ivv + qm * qn * Jvv;
        }
        if (qs_n != 0.0) z += qm * qs_n * volface(c, t, n);
    }
    if (qs_m != 0.0) {
        for (int q = 0; q < 2; ++q) {
            const int tp = c->ftet[2 * n + q];
            if (tp < 0) continue;
            const double sp = q == 0 ? 1.0 : -1.0;
            const double qn = -c->kappa[tp] * sp * c->farea[n] / c->tvol[tp];
            z += qs_m * qn * volface(c, tp, m);   /* = Int_{face m} Int_{tp} G, tetrahedron outer */
        }
        if (qs_n != 0.0) z += qs_m * qs_n * faceface(c, m, n);
    }
    return z;
}

static zc vmo_entry_cb(const void *c, int m, int n) { return vmo_entry((const vmo_ctx *)c, m, n); }

void vmo_fill(const vmo_ctx *c, const int32_t *rows, int nr, const int32_t *cols, int nc, zc *out)
{
#pragma omp parallel for schedule(dynamic, 16) collapse(2)
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nc; ++j) out[(int64_t)i * nc + j] = vmo_entry(c, rows[i], cols[j]);
}

/* b[r*nf + m] = Int kappa f_m . p_hat exp(-jk k_hat . r) dV */
void vmo_rhs(const vmo_ctx *c, int nrhs, const double *khat, const double *phat, zc *b)
{
#pragma omp parallel for schedule(static)
    for (int m = 0; m < c->nf; ++m)
        for (int r = 0; r < nrhs; ++r) {
            zc acc = 0.0;
            for (int p = 0; p < 2; ++p) {
                const int t = c->ftet[2 * m + p];
                if (t < 0) continue;
                const double s = p == 0 ? 1.0 : -1.0;
                const double *v = c->xyz + 3 * c->ffree[2 * m + p];
                const double cm = s * c->farea[m] / (3.0 * c->tvol[t]) * c->kappa[t] * c->tvol[t];
                for (int q = 0; q < NQT; ++q) {
                    const double *rq = c->tqp + (t * NQT + q) * 3;
                    double a[3];
                    sub3(rq, v, a);
                    acc += cm * c->tw[q] * dot3(a, phat + 3 * r) * cexp(-I * c->k * dot3(khat + 3 * r, rq));
                }
            }
            b[(int64_t)r * c->nf + m] = acc;
        }
}

/* P(r_hat) = Int kappa D/eps0 exp(+jk r_hat . r') dV' = sum_n x_n Int kappa f_n exp(...) */
void vmo_radiation(const vmo_ctx *c, const zc *x, int ndir, const double *rhat, zc *P)
{
#pragma omp parallel for schedule(static)
    for (int dd = 0; dd < ndir; ++dd) {
        zc acc[3] = {0, 0, 0};
        for (int n = 0; n < c->nf; ++n)
            for (int p = 0; p < 2; ++p) {
                const int t = c->ftet[2 * n + p];
                if (t < 0) continue;
                const double s = p == 0 ? 1.0 : -1.0;
                const double *v = c->xyz + 3 * c->ffree[2 * n + p];
                const zc cn = x[n] * s * c->farea[n] / 3.0 * c->kappa[t];
                for (int q = 0; q < NQT; ++q) {
                    const double *rq = c->tqp + (t * NQT + q) * 3;
                    const zc ph = cn * c->tw[q] * cexp(I * c->k * dot3(rhat + 3 * dd, rq));
                    acc[0] += ph * (rq[0] - v[0]);
                    acc[1] += ph * (rq[1] - v[1]);
                    acc[2] += ph * (rq[2] - v[2]);
                }
            }
        P[3 * dd] = acc[0]; P[3 * dd + 1] = acc[1]; P[3 * dd + 2] = acc[2];
    }
}

void vmo_aca_many(const vmo_ctx *c, int nb, const int32_t *idx, const int64_t *roff, const int32_t *m,
                  const int64_t *coff, const int32_t *n, double tol, const int32_t *kmax, const int64_t *uoff,
                  const int64_t *voff, zc *U, zc *V, int32_t *rank)
{
    hmo_aca_many_generic(vmo_entry_cb, c, nb, idx, roff, m, coff, n, tol, kmax, uoff, voff, U, V, rank);
}

int vmo_aca(const vmo_ctx *c, const int32_t *rows, int m, const int32_t *cols, int n, double tol, int kmax, zc *U,
            zc *V)
{
    return hmo_aca_generic(vmo_entry_cb, c, rows, m, cols, n, tol, kmax, U, V);
}
