/*
 * CPU oracle, complex128 — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  The product (CUDA) path shares no code with it.
 *
 * What it computes (arxiv 2307.03968 §II, eqs. 1-5; §III, eqs. 6-7):
 *   - Galerkin S-EFIE entries for RWG basis functions (§II, eq. 3 tested with
 *     RWG functions, giving Z of eq. 5), time convention e^{jwt},
 *     G(R) = exp(-jkR) / (4 pi R):
 *         Z_mn = jk eta  Int_Tm Int_Tn [ f_m . f_n - (div f_m)(div' f_n)/k^2 ] G dS' dS
 *     RWG function on T+ / T-:  f = +-(l / 2A) (r - v_free),  div f = +-l/A.
 *   - Right-hand side b_m = Int f_m . E_inc dS for a plane wave
 *     E_inc = p_hat exp(-jk k_hat . r)   (eq. 5, "b is a known incident plane wave").
 *   - Far-field radiation vector F(r_hat) = Int J exp(+jk r_hat . r') dS' of the
 *     current J = sum_n x_n f_n, for the bistatic RCS of the paper's Figs. 2-4.
 *   - Partially pivoted adaptive cross approximation of a far block (§III,
 *     "Z_sub(m x n) ~ U(m x k) V(k x n)", ACA of refs. [22,23] = Bebendorf 2000).
 *
 * Quadrature: the 7-point degree-5 rule on triangles (Radon 1948; Hammer,
 * Marlowe & Stroud 1956), points given in closed form below.
 * Singular / near-singular pairs: the 1/R part of G is integrated analytically
 * over the source triangle (Wilton, Rao, Glisson et al., IEEE TAP 1984; Graglia,
 * IEEE TAP 1993) and only the smooth remainder (exp(-jkR)-1)/(4 pi R) is
 * integrated by quadrature.  A triangle pair is treated this way when the
 * distance between centroids is below 2 x the larger maximum edge length of the
 * two triangles (the paper is silent on quadrature; this is the build's reading).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zc;

#define NQ 7
#define EXTRACT_FACTOR 2.0

typedef struct {
    int nv, nt, ne;
    const double *xyz;      /* nv x 3 */
    const int32_t *tri;     /* nt x 3 */
    const int32_t *etri;    /* ne x 2 : T+, T- */
    const int32_t *efree;   /* ne x 2 : free vertex of T+, of T- */
    const double *elen;     /* ne : edge length */
    double k, eta;
    /* per-triangle derived data */
    double *area, *cen, *hmax, *qp, *nrm; /* nt, nt*3, nt, nt*NQ*3, nt*3 */
    double qw[NQ];
} hmo_ctx;

static void quad_rule(double bary[NQ][3], double w[NQ])
{
    const double s15 = sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
    const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
    const double w0 = 9.0 / 40.0, w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    double pts[NQ][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                         {a1, a1, b1}, {a1, b1, a1}, {b1, a1, a1},
                         {a2, a2, b2}, {a2, b2, a2}, {b2, a2, a2}};
    double ww[NQ] = {w0, w1, w1, w1, w2, w2, w2};
    memcpy(bary, pts, sizeof(pts));
    memcpy(w, ww, sizeof(ww));
}

static inline void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double norm3(const double *a) { return sqrt(dot3(a, a)); }

hmo_ctx *hmo_ctx_new(int nv, const double *xyz, int nt, const int32_t *tri, int ne,
                     const int32_t *etri, const int32_t *efree, const double *elen,
                     double k, double eta)
{
    hmo_ctx *c = (hmo_ctx *)calloc(1, sizeof(hmo_ctx));
    c->nv = nv; c->nt = nt; c->ne = ne;
    c->xyz = xyz; c->tri = tri; c->etri = etri; c->efree = efree; c->elen = elen;
    c->k = k; c->eta = eta;
    c->area = (double *)malloc(sizeof(double) * nt);
    c->cen = (double *)malloc(sizeof(double) * nt * 3);
    c->hmax = (double *)malloc(sizeof(double) * nt);
    c->qp = (double *)malloc(sizeof(double) * nt * NQ * 3);
    c->nrm = (double *)malloc(sizeof(double) * nt * 3);
    double bary[NQ][3];
    quad_rule(bary, c->qw);
    for (int t = 0; t < nt; ++t) {
        const double *p0 = xyz + 3 * tri[3 * t], *p1 = xyz + 3 * tri[3 * t + 1], *p2 = xyz + 3 * tri[3 * t + 2];
        double e1[3], e2[3], e3[3], n[3];
        sub3(p1, p0, e1); sub3(p2, p0, e2); sub3(p2, p1, e3);
        cross3(e1, e2, n);
        double nn = norm3(n);
        c->area[t] = 0.5 * nn;
        for (int d = 0; d < 3; ++d) {
            c->nrm[3 * t + d] = n[d] / nn;
            c->cen[3 * t + d] = (p0[d] + p1[d] + p2[d]) / 3.0;
        }
        double h = norm3(e1);
        if (norm3(e2) > h) h = norm3(e2);
        if (norm3(e3) > h) h = norm3(e3);
        c->hmax[t] = h;
        for (int q = 0; q < NQ; ++q)
            for (int d = 0; d < 3; ++d)
                c->qp[(t * NQ + q) * 3 + d] = bary[q][0] * p0[d] + bary[q][1] * p1[d] + bary[q][2] * p2[d];
    }
    return c;
}

void hmo_ctx_free(hmo_ctx *c)
{
    if (!c) return;
    free(c->area); free(c->cen); free(c->hmax); free(c->qp); free(c->nrm);
    free(c);
}

/*
 * Potential integrals of the 1/R kernel over a flat triangle (Wilton et al.
 * 1984, eqs. for a uniform and a linear source on a polygon):
 *   s0      = Int_T 1/|r - r'| dS'
 *   s1v     = Int_T (rho' - rho)/|r - r'| dS'     (in-plane vector)
 *   sR      = Int_T |r - r'| dS'                  (if sR_out is not NULL)
 * where rho is the projection of r onto the triangle's plane.  sR follows from
 * the in-plane divergence of (rho' - rho) R, which is 3R - d^2/R:
 *   sR = ( d^2 s0 + sum_edges t * Int_edge R dl ) / 3,
 *   Int_edge R dl = ( l+ R+ - l- R- + R0^2 f ) / 2.
 * Edges are taken counter-clockwise about the unit normal n; for each edge,
 * l_hat is its direction, u_hat = l_hat x n the outward in-plane normal,
 * t = signed distance from rho to the edge line (positive inside),
 * l+- the coordinates of the edge end points along l_hat relative to rho,
 * R0^2 = t^2 + d^2 and R+- = sqrt(R0^2 + l+-^2).
 */
void hmo_potential_integrals3(const double *p0, const double *p1, const double *p2,
                              const double *r, double *s0_out, double *s1v_out, double *sR_out)
{
    const double *P[3] = {p0, p1, p2};
    double e1[3], e2[3], n[3];
    sub3(p1, p0, e1); sub3(p2, p0, e2); cross3(e1, e2, n);
    double nn = norm3(n);
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    double rp0[3];
    sub3(r, p0, rp0);
    double d = dot3(n, rp0);
    double ad = fabs(d);
    double rho[3] = {r[0] - d * n[0], r[1] - d * n[1], r[2] - d * n[2]};
    double s0 = 0.0, s1[3] = {0, 0, 0}, edgeR = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double *a = P[i], *b = P[(i + 1) % 3];
        double lv[3];
        sub3(b, a, lv);
        double ll = norm3(lv);
        double lh[3] = {lv[0] / ll, lv[1] / ll, lv[2] / ll};
        double uh[3];
        cross3(lh, n, uh);
        double am[3], bm[3];
        sub3(a, rho, am); sub3(b, rho, bm);
        double lp = dot3(bm, lh), lm = dot3(am, lh);
        double t = dot3(am, uh); /* positive when rho is on the interior side of the edge */
        double R02 = t * t + d * d;
        double Rp = sqrt(R02 + lp * lp), Rm = sqrt(R02 + lm * lm);
        double f;
        if (lm < 0.0 && lp < 0.0)
            f = log((Rm - lm) / (Rp - lp));
        else
            f = log((Rp + lp) / (Rm + lm));
        if (R02 > 0.0) {
            double term = t * f;
            if (ad > 0.0)
                term -= ad * (atan(t * lp / (R02 + ad * Rp)) - atan(t * lm / (R02 + ad * Rm)));
            s0 += term;
        }
        double g = 0.5 * ((R02 > 0.0 ? R02 * f : 0.0) + lp * Rp - lm * Rm);
        /* u_hat points outward; the vector integral uses the outward normal */
        s1[0] += g * uh[0]; s1[1] += g * uh[1]; s1[2] += g * uh[2];
        edgeR += t * g;   /* g is also Int_edge R dl */
    }
    *s0_out = s0;
    s1v_out[0] = s1[0]; s1v_out[1] = s1[1]; s1v_out[2] = s1[2];
    if (sR_out) *sR_out = (d * d * s0 + edgeR) / 3.0;
}

void hmo_potential_integrals(const double *p0, const double *p1, const double *p2,
                             const double *r, double *s0_out, double *s1v_out)
{
    hmo_potential_integrals3(p0, p1, p2, r, s0_out, s1v_out, NULL);
}

/* (1/(A_m A_n)) Int_Tm Int_Tn [ 1/4 (r - vm).(r' - vn) - 1/k^2 ] G dS' dS */
static zc pair_integral(const hmo_ctx *c, int tm, const double *vm, int tn, const double *vn)
{
    const double k = c->k, ik2 = 1.0 / (c->k * c->k);
    const double inv4pi = 1.0 / (4.0 * M_PI);
    double dc[3];
    sub3(c->cen + 3 * tm, c->cen + 3 * tn, dc);
    double h = c->hmax[tm] > c->hmax[tn] ? c->hmax[tm] : c->hmax[tn];
    int extract = dot3(dc, dc) < (EXTRACT_FACTOR * h) * (EXTRACT_FACTOR * h);
    zc acc = 0.0;
    for (int i = 0; i < NQ; ++i) {
        const double *ri = c->qp + (tm * NQ + i) * 3;
        double a[3];
        sub3(ri, vm, a);
        zc inner = 0.0;
        for (int j = 0; j < NQ; ++j) {
            const double *rj = c->qp + (tn * NQ + j) * 3;
            double bj[3], dr[3];
            sub3(rj, vn, bj);
            sub3(ri, rj, dr);
            double R = norm3(dr);
            double fac = 0.25 * dot3(a, bj) - ik2;
            zc g;
            if (extract) {
                if (R < 1e-14) g = -I * k * inv4pi;
                else {
                    double sh = sin(0.5 * k * R);
                    g = (-2.0 * sh * sh - I * sin(k * R)) * inv4pi / R;
                }
            } else {
                g = cexp(-I * k * R) * inv4pi / R;
            }
            inner += c->qw[j] * fac * g;
        }
        if (extract) {
            const int *tv = c->tri + 3 * tn;
            double s0, s1v[3];
            hmo_potential_integrals(c->xyz + 3 * tv[0], c->xyz + 3 * tv[1], c->xyz + 3 * tv[2], ri, &s0, s1v);
            /* S1 = Int (r' - vn)/R = s1v + (rho - vn) s0, rho = projection of ri */
            const double *nrm = c->nrm + 3 * tn;
            double rv[3];
            sub3(ri, c->xyz + 3 * tv[0], rv);
            double d = dot3(nrm, rv);
            double rho_m_vn[3] = {ri[0] - d * nrm[0] - vn[0], ri[1] - d * nrm[1] - vn[1], ri[2] - d * nrm[2] - vn[2]};
            double S1[3] = {s1v[0] + rho_m_vn[0] * s0, s1v[1] + rho_m_vn[1] * s0, s1v[2] + rho_m_vn[2] * s0};
            inner += (0.25 * dot3(a, S1) - ik2 * s0) * inv4pi / c->area[tn];
        }
        acc += c->qw[i] * inner;
    }
    return acc;
}

zc hmo_entry(const hmo_ctx *c, int m, int n)
{
    zc z = 0.0;
    for (int p = 0; p < 2; ++p) {
        int tm = c->etri[2 * m + p];
        const double *vm = c->xyz + 3 * c->efree[2 * m + p];
        double sp = p == 0 ? 1.0 : -1.0;
        for (int q = 0; q < 2; ++q) {
            int tn = c->etri[2 * n + q];
            const double *vn = c->xyz + 3 * c->efree[2 * n + q];
            double sq = q == 0 ? 1.0 : -1.0;
            z += sp * sq * pair_integral(c, tm, vm, tn, vn);
        }
    }
    return I * c->k * c->eta * c->elen[m] * c->elen[n] * z;
}

/* The quadrature rule, for tests: bary[7*3], w[7]. */
void hmo_quad_rule(double *bary, double *w) { quad_rule((double (*)[3])bary, w); }

/* out[i*nc + j] = Z[rows[i], cols[j]] */
void hmo_fill(const hmo_ctx *c, const int32_t *rows, int nr, const int32_t *cols, int nc, zc *out)
{
#pragma omp parallel for schedule(dynamic, 16) collapse(2)
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nc; ++j)
            out[(int64_t)i * nc + j] = hmo_entry(c, rows[i], cols[j]);
}

/* b[r*ne + m] = Int f_m . p_hat_r exp(-jk k_hat_r . r) dS, for nrhs plane waves */
void hmo_rhs(const hmo_ctx *c, int nrhs, const double *khat, const double *phat, zc *b)
{
#pragma omp parallel for schedule(static)
    for (int m = 0; m < c->ne; ++m) {
        for (int r = 0; r < nrhs; ++r) {
            const double *kh = khat + 3 * r, *ph = phat + 3 * r;
            zc acc = 0.0;
            for (int p = 0; p < 2; ++p) {
                int t = c->etri[2 * m + p];
                const double *v = c->xyz + 3 * c->efree[2 * m + p];
                double s = p == 0 ? 1.0 : -1.0;
                for (int q = 0; q < NQ; ++q) {
                    const double *rq = c->qp + (t * NQ + q) * 3;
                    double a[3];
                    sub3(rq, v, a);
                    acc += s * c->qw[q] * dot3(a, ph) * cexp(-I * c->k * dot3(kh, rq));
                }
            }
            b[(int64_t)r * c->ne + m] = 0.5 * c->elen[m] * acc;
        }
    }
}

/* F[3*d + :] = Int J(r') exp(+jk rhat_d . r') dS', J = sum_n x[n] f_n */
void hmo_radiation(const hmo_ctx *c, const zc *x, int ndir, const double *rhat, zc *F)
{
#pragma omp parallel for schedule(static)
    for (int dd = 0; dd < ndir; ++dd) {
        const double *rh = rhat + 3 * dd;
        zc f[3] = {0, 0, 0};
        for (int n = 0; n < c->ne; ++n) {
            for (int p = 0; p < 2; ++p) {
                int t = c->etri[2 * n + p];
                const double *v = c->xyz + 3 * c->efree[2 * n + p];
                double s = p == 0 ? 1.0 : -1.0;
                for (int q = 0; q < NQ; ++q) {
                    const double *rq = c->qp + (t * NQ + q) * 3;
                    zc ph = x[n] * s * 0.5 * c->elen[n] * c->qw[q] * cexp(I * c->k * dot3(rh, rq));
                    f[0] += ph * (rq[0] - v[0]);
                    f[1] += ph * (rq[1] - v[1]);
                    f[2] += ph * (rq[2] - v[2]);
                }
            }
        }
        F[3 * dd] = f[0]; F[3 * dd + 1] = f[1]; F[3 * dd + 2] = f[2];
    }
}

/*
 * Partially pivoted ACA (Bebendorf 2000) of the block Z[rows, cols]:
 *   Z ~ sum_l u_l v_l^T,  U = [u_0 .. u_{k-1}] (m x k), V = [v_0; ..; v_{k-1}] (k x n).
 * Step: take row i* of the residual, pivot column j* = argmax |row|, scale the row
 * by the pivot to get v, take column j* of the residual as u, then pick the next
 * row as the largest |u_i| among unused rows.  Stop when |u_k| |v_k| <= tol |S_k|_F
 * with |S_k|_F^2 updated incrementally.  U is stored column-major (U[l*m + i]),
 * V row-major (V[l*n + j]).  Returns the rank k (<= kmax).
 */
typedef zc (*hmo_entry_fn)(const void *ctx, int m, int n);

int hmo_aca_generic(hmo_entry_fn entry, const void *c, const int32_t *rows, int m, const int32_t *cols, int n,
                    double tol, int kmax, zc *U, zc *V)
{
    char *used = (char *)calloc(m, 1);
    zc *row = (zc *)malloc(sizeof(zc) * n);
    double s2 = 0.0;
    int k = 0, istar = 0;
    if (kmax > m) kmax = m;
    if (kmax > n) kmax = n;
    while (k < kmax) {
        for (int j = 0; j < n; ++j) {
            zc v = entry(c, rows[istar], cols[j]);
            for (int l = 0; l < k; ++l) v -= U[(int64_t)l * m + istar] * V[(int64_t)l * n + j];
            row[j] = v;
        }
        used[istar] = 1;
        int jstar = 0;
        double best = -1.0;
        for (int j = 0; j < n; ++j) {
            double a = cabs(row[j]);
            if (a > best) { best = a; jstar = j; }
        }
        if (best <= 0.0) {
            int next = -1;
            for (int i = 0; i < m; ++i) if (!used[i]) { next = i; break; }
            if (next < 0) break;
            istar = next;
            continue;
        }
        zc piv = row[jstar];
        zc *v = V + (int64_t)k * n, *u = U + (int64_t)k * m;
        for (int j = 0; j < n; ++j) v[j] = row[j] / piv;
        for (int i = 0; i < m; ++i) {
            zc w = entry(c, rows[i], cols[jstar]);
            for (int l = 0; l < k; ++l) w -= V[(int64_t)l * n + jstar] * U[(int64_t)l * m + i];
            u[i] = w;
        }
        double nu2 = 0.0, nv2 = 0.0;
        for (int i = 0; i < m; ++i) nu2 += creal(u[i] * conj(u[i]));
        for (int j = 0; j < n; ++j) nv2 += creal(v[j] * conj(v[j]));
        zc cross = 0.0;
        for (int l = 0; l < k; ++l) {
            zc uu = 0.0, vv = 0.0;
            for (int i = 0; i < m; ++i) uu += conj(U[(int64_t)l * m + i]) * u[i];
            for (int j = 0; j < n; ++j) vv += conj(V[(int64_t)l * n + j]) * v[j];
            cross += uu * vv;
        }
        s2 += 2.0 * creal(cross) + nu2 * nv2;
        ++k;
        if (sqrt(nu2 * nv2) <= tol * sqrt(s2)) break;
        int next = -1;
        double bu = -1.0;
        for (int i = 0; i < m; ++i) {
            if (used[i]) continue;
            double a = cabs(u[i]);
            if (a > bu) { bu = a; next = i; }
        }
        if (next < 0) break;
        istar = next;
    }
    free(used);
    free(row);
    return k;
}

static zc rwg_entry_cb(const void *c, int m, int n) { return hmo_entry((const hmo_ctx *)c, m, n); }

int hmo_aca(const hmo_ctx *c, const int32_t *rows, int m, const int32_t *cols, int n,
            double tol, int kmax, zc *U, zc *V)
{
    return hmo_aca_generic(rwg_entry_cb, c, rows, m, cols, n, tol, kmax, U, V);
}

void hmo_aca_many_generic(hmo_entry_fn entry, const void *c, int nb, const int32_t *idx, const int64_t *roff,
                          const int32_t *m, const int64_t *coff, const int32_t *n, double tol, const int32_t *kmax,
                          const int64_t *uoff, const int64_t *voff, zc *U, zc *V, int32_t *rank)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nb; ++b)
        rank[b] = hmo_aca_generic(entry, c, idx + roff[b], m[b], idx + coff[b], n[b], tol, kmax[b], U + uoff[b],
                                  V + voff[b]);
}

/* ACA of many blocks in parallel; block b covers rows[roff[b] .. roff[b]+m[b]),
 * cols[coff[b] .. coff[b]+n[b]); U/V written at uoff[b]/voff[b] with room for
 * kmax[b] terms.  rank[b] receives the rank. */
void hmo_aca_many(const hmo_ctx *c, int nb, const int32_t *idx, const int64_t *roff, const int32_t *m,
                  const int64_t *coff, const int32_t *n, double tol, const int32_t *kmax,
                  const int64_t *uoff, const int64_t *voff, zc *U, zc *V, int32_t *rank)
{
    hmo_aca_many_generic(rwg_entry_cb, c, nb, idx, roff, m, coff, n, tol, kmax, uoff, voff, U, V, rank);
}
