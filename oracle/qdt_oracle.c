/*
 * qdt_oracle.c -- plain, slow FP64 CPU oracle for the AO integrals of the
 * quaternion Dirac-Coulomb-Breit AO->MO transformation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA path and uses a different algorithm (Obara-Saika vertical and
 * Head-Gordon-Pople horizontal recursions here; McMurchie-Davidson there).
 *
 * What it computes (paper Sec. 2.1-2.3):
 *   - scalar two-electron integrals (ab|cd) over the large-component basis
 *     chi_mu (contracted Cartesian Gaussians, every Cartesian component
 *     normalised on its own) and over the small-component derivative basis
 *     d/dr_K chi_mu (index 3 mu + K), kernel 1/r12 (Eqs. Coulomb and DCInt);
 *   - the gauge-kernel integrals (ab| r12_I r12_J / r12^3 |cd) of
 *     Eq. gaugeInt, as  delta_IJ (ab|1/r12|cd) - (ab| d_I d_J r12 |cd), the
 *     second term being the double centre derivative
 *     (d_A + d_B)_I (d_A + d_B)_J (ab|r12|cd)   (translational invariance);
 *   - Schwarz diagonals (ab|ab) for Eq. SchwarzDen.
 *
 * Kernel-generic Obara-Saika: the vertical recursion only needs the
 * (ss|ss)^(m) auxiliaries Theta * G_m(T) with dG_m/dT = -G_{m+1}:
 *   1/r12 : Theta = 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD,   G_m = F_m
 *   r12   : Theta = (pi^2/(p q))^{3/2} / sqrt(pi rho) K_AB K_CD,
 *           G_m = F_m - F_{m-1},   F_{-1}(T) = -(2 T F_0(T) + exp(-T)),
 * the r12 base being the Gaussian-smeared distance
 * <|R+u|> = ((1+2T) F_0(T) + exp(-T)) / sqrt(pi rho),  T = rho R^2.
 * Both are pinned in the tests (closed forms, radial quadrature, finite
 * differences in the centres and the trace identity sum_I K_II = 1/r12).
 */
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <string.h>

#define OR_MAXLT 18          /* max total order of a triple table            */
#define OR_MAXM 48           /* max Boys order                               */

/* ------------------------------------------------------------------ Boys */

/* F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt for m = 0..mmax. */
void or_boys(double T, int mmax, double *F)
{
    if (T < 45.0) {
        /* series for the top order, then the stable downward recursion
           F_m = (2T F_{m+1} + e^{-T}) / (2m+1). */
        int M = mmax;
        double term = 1.0 / (2.0 * M + 1.0), sum = term;
        for (int k = 1; k < 1000; ++k) {
            term *= 2.0 * T / (2.0 * M + 2.0 * k + 1.0);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        double et = exp(-T);
        F[M] = et * sum;
        for (int m = M - 1; m >= 0; --m)
            F[m] = (2.0 * T * F[m + 1] + et) / (2.0 * m + 1.0);
    } else {
        /* F_0 from erf, then upward recursion (stable for large T). */
        double et = exp(-T);
        F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
        for (int m = 0; m < mmax; ++m)
            F[m + 1] = ((2.0 * m + 1.0) * F[m] - et) / (2.0 * T);
    }
}

double or_boys_minus1(double T)
{
    double F[1];
    or_boys(T, 0, F);
    return -(2.0 * T * F[0] + exp(-T));
}

/* G_m(T): kernel 0 = 1/r12 (F_m), kernel 1 = r12 (F_m - F_{m-1}). */
static void kernel_aux(int kernel, double T, int mmax, double *G)
{
    double F[OR_MAXM + 2];
    or_boys(T, mmax, F);
    if (kernel == 0) {
        for (int m = 0; m <= mmax; ++m) G[m] = F[m];
    } else {
        double Fm1 = -(2.0 * T * F[0] + exp(-T));
        G[0] = F[0] - Fm1;
        for (int m = 1; m <= mmax; ++m) G[m] = F[m] - F[m - 1];
    }
}

/* ------------------------------------------------------ Cartesian tables */

static int ntri(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }  /* triples with order <= L */
static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* position of (i,j,k) among all triples, ordered by total order then x-major */
static int tidx(int i, int j, int k)
{
    int l = i + j + k, jk = j + k;
    return l * (l + 1) * (l + 2) / 6 + jk * (jk + 1) / 2 + k;
}

static int g_tri[1330][3];   /* ntri(OR_MAXLT) = 1330 */
static int g_tri_ready = 0;

static void tri_init(void)
{
    if (g_tri_ready) return;
    for (int l = 0; l <= OR_MAXLT; ++l)
        for (int i = l; i >= 0; --i)
            for (int j = l - i; j >= 0; --j) {
                int k = l - i - j, t = tidx(i, j, k);
                g_tri[t][0] = i; g_tri[t][1] = j; g_tri[t][2] = k;
            }
    g_tri_ready = 1;
}

static int tri_l(int t) { return g_tri[t][0] + g_tri[t][1] + g_tri[t][2]; }
static int tri_step(int t, int dir, int delta)
{
    int v[3] = {g_tri[t][0], g_tri[t][1], g_tri[t][2]};
    v[dir] += delta;
    if (v[dir] < 0) return -1;
    return tidx(v[0], v[1], v[2]);
}
static int tri_dir(int t) { return g_tri[t][0] ? 0 : (g_tri[t][1] ? 1 : 2); }

/* ------------------------------------------- primitive quartet (OS + HGP) */

/*
 * All integrals over primitive Cartesian Gaussians
 *   g_a = (x-A_x)^ax (y-A_y)^ay (z-A_z)^az exp(-alpha |r-A|^2)   (unnormalised)
 * for every triple a with |a| <= La, b <= Lb, c <= Lc, d <= Ld.
 * out[ntri(La)][ntri(Lb)][ntri(Lc)][ntri(Ld)].
 */
void or_prim_cum(int kernel,
                 const double *A, double al, int La, const double *B, double be, int Lb,
                 const double *C, double ga, int Lc, const double *D, double de, int Ld,
                 double *out)
{
    tri_init();
    double p = al + be, q = ga + de, rho = p * q / (p + q);
    double P[3], Q[3], PA[3], PQ[3], QC[3], AB[3], CD[3];
    double rab2 = 0, rcd2 = 0, rpq2 = 0;
    for (int i = 0; i < 3; ++i) {
        P[i] = (al * A[i] + be * B[i]) / p;
        Q[i] = (ga * C[i] + de * D[i]) / q;
        PA[i] = P[i] - A[i]; QC[i] = Q[i] - C[i]; PQ[i] = P[i] - Q[i];
        AB[i] = A[i] - B[i]; CD[i] = C[i] - D[i];
        rab2 += AB[i] * AB[i]; rcd2 += CD[i] * CD[i]; rpq2 += PQ[i] * PQ[i];
    }
    double Kab = exp(-al * be / p * rab2), Kcd = exp(-ga * de / q * rcd2);
    double T = rho * rpq2, theta;
    if (kernel == 0)
        theta = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * Kab * Kcd;
    else
        theta = pow(M_PI * M_PI / (p * q), 1.5) / sqrt(M_PI * rho) * Kab * Kcd;

    int Le = La + Lb, Lf = Lc + Ld, Mt = Le + Lf;
    int ne = ntri(Le), nf = ntri(Lf), nm = Mt + 1;
    double G[OR_MAXM + 2];
    kernel_aux(kernel, T, Mt, G);

    /* vertical recursion V[m][e][f] */
    double *V = (double *)calloc((size_t)nm * ne * nf, sizeof(double));
#define VV(m, e, f) V[((size_t)(m) * ne + (e)) * nf + (f)]
    for (int m = 0; m <= Mt; ++m) VV(m, 0, 0) = theta * G[m];
    for (int e = 1; e < ne; ++e) {
        int i = tri_dir(e), e1 = tri_step(e, i, -1), e2 = tri_step(e1, i, -1);
        double ei1 = g_tri[e1][i];
        for (int m = 0; m <= Mt - tri_l(e); ++m) {
            double v = PA[i] * VV(m, e1, 0) - rho / p * PQ[i] * VV(m + 1, e1, 0);
            if (e2 >= 0) v += ei1 / (2.0 * p) * (VV(m, e2, 0) - rho / p * VV(m + 1, e2, 0));
            VV(m, e, 0) = v;
        }
    }
    for (int f = 1; f < nf; ++f) {
        int i = tri_dir(f), f1 = tri_step(f, i, -1), f2 = tri_step(f1, i, -1);
        double fi1 = g_tri[f1][i];
        for (int e = 0; e < ne; ++e) {
            int em = tri_step(e, i, -1);
            double ei = g_tri[e][i];
            for (int m = 0; m <= Mt - tri_l(e) - tri_l(f); ++m) {
                double v = QC[i] * VV(m, e, f1) + rho / q * PQ[i] * VV(m + 1, e, f1);
                if (f2 >= 0) v += fi1 / (2.0 * q) * (VV(m, e, f2) - rho / q * VV(m + 1, e, f2));
                if (em >= 0) v += ei / (2.0 * (p + q)) * VV(m + 1, em, f1);
                VV(m, e, f) = v;
            }
        }
    }

    /* horizontal recursion on the bra: (a, b+1_i| = (a+1_i, b| + AB_i (a, b| */
    int nA = ntri(La), nB = ntri(Lb), nC = ntri(Lc), nD = ntri(Ld);
    double *H = (double *)malloc((size_t)nA * nB * nf * sizeof(double));
    double *X = (double *)malloc((size_t)ne * nB * sizeof(double));
    for (int f = 0; f < nf; ++f) {
        for (int e = 0; e < ne; ++e) X[e * nB] = VV(0, e, f);
        for (int b = 1; b < nB; ++b) {
            int i = tri_dir(b), b1 = tri_step(b, i, -1);
            for (int a = 0; a < ntri(Le - tri_l(b)); ++a)
                X[a * nB + b] = X[tri_step(a, i, 1) * nB + b1] + AB[i] * X[a * nB + b1];
        }
        for (int a = 0; a < nA; ++a)
            for (int b = 0; b < nB; ++b)
                H[((size_t)a * nB + b) * nf + f] = X[a * nB + b];
    }
    free(X);
    /* horizontal recursion on the ket */
    double *Y = (double *)malloc((size_t)nf * nD * sizeof(double));
    for (int a = 0; a < nA; ++a)
        for (int b = 0; b < nB; ++b) {
            const double *h = H + ((size_t)a * nB + b) * nf;
            for (int f = 0; f < nf; ++f) Y[f * nD] = h[f];
            for (int d = 1; d < nD; ++d) {
                int i = tri_dir(d), d1 = tri_step(d, i, -1);
                for (int c = 0; c < ntri(Lf - tri_l(d)); ++c)
                    Y[c * nD + d] = Y[tri_step(c, i, 1) * nD + d1] + CD[i] * Y[c * nD + d1];
            }
            double *o = out + ((size_t)a * nB + b) * nC * nD;
            for (int c = 0; c < nC; ++c)
                for (int d = 0; d < nD; ++d) o[c * nD + d] = Y[c * nD + d];
        }
    free(Y); free(H); free(V);
#undef VV
}

/* Exact-order primitive block out[ncart(la)][ncart(lb)][ncart(lc)][ncart(ld)]. */
void or_prim_block(int kernel,
                   const double *A, double al, int la, const double *B, double be, int lb,
                   const double *C, double ga, int lc, const double *D, double de, int ld,
                   double *out)
{
    int nA = ntri(la), nB = ntri(lb), nC = ntri(lc), nD = ntri(ld);
    double *cum = (double *)malloc((size_t)nA * nB * nC * nD * sizeof(double));
    or_prim_cum(kernel, A, al, la, B, be, lb, C, ga, lc, D, de, ld, cum);
    int oa = ntri(la - 1), ob = ntri(lb - 1), oc = ntri(lc - 1), od = ntri(ld - 1);
    int ca = ncart(la), cb = ncart(lb), cc = ncart(lc), cd = ncart(ld);
    if (la == 0) oa = 0;
    if (lb == 0) ob = 0;
    if (lc == 0) oc = 0;
    if (ld == 0) od = 0;
    for (int a = 0; a < ca; ++a)
        for (int b = 0; b < cb; ++b)
            for (int c = 0; c < cc; ++c)
                for (int d = 0; d < cd; ++d)
                    out[((a * cb + b) * cc + c) * cd + d] =
                        cum[(((size_t)(oa + a) * nB + ob + b) * nC + oc + c) * nD + od + d];
    free(cum);
}

/* ----------------------------------------------------- centre derivatives */

typedef struct { double w; int a, b; } DTerm;

/* apply (d/dA_I + d/dB_I) to a list of bra terms;
   d/dA_I g_a = 2 alpha g_{a+1_I} - a_I g_{a-1_I}. */
static int dterm_apply(const DTerm *in, int n, DTerm *out, int I, double al, double be)
{
    int k = 0;
    for (int t = 0; t < n; ++t) {
        int a = in[t].a, b = in[t].b;
        out[k++] = (DTerm){in[t].w * 2.0 * al, tri_step(a, I, 1), b};
        if (g_tri[a][I] > 0) out[k++] = (DTerm){-in[t].w * g_tri[a][I], tri_step(a, I, -1), b};
        out[k++] = (DTerm){in[t].w * 2.0 * be, a, tri_step(b, I, 1)};
        if (g_tri[b][I] > 0) out[k++] = (DTerm){-in[t].w * g_tri[b][I], a, tri_step(b, I, -1)};
    }
    return k;
}

static const int IJ6[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};

/*
 * Primitive blocks of (ab| d_I d_J r12 |cd), IJ in xx,xy,xz,yy,yz,zz:
 * out[6][ncart(la)][ncart(lb)][ncart(lc)][ncart(ld)].
 * form 1: (d_A+d_B)_I (d_A+d_B)_J (ab|r12|cd)
 * form 2: -(d_A+d_B)_I (d_C+d_D)_J (ab|r12|cd)
 */
void or_prim_ddr(int form,
                 const double *A, double al, int la, const double *B, double be, int lb,
                 const double *C, double ga, int lc, const double *D, double de, int ld,
                 double *out)
{
    tri_init();
    int La = la + (form == 1 ? 2 : 1), Lb = lb + (form == 1 ? 2 : 1);
    int Lc = lc + (form == 1 ? 0 : 1), Ld = ld + (form == 1 ? 0 : 1);
    int nA = ntri(La), nB = ntri(Lb), nC = ntri(Lc), nD = ntri(Ld);
    double *cum = (double *)malloc((size_t)nA * nB * nC * nD * sizeof(double));
    or_prim_cum(1, A, al, La, B, be, Lb, C, ga, Lc, D, de, Ld, cum);
#define CUM(a, b, c, d) cum[(((size_t)(a) * nB + (b)) * nC + (c)) * nD + (d)]
    int ca = ncart(la), cb = ncart(lb), cc = ncart(lc), cd = ncart(ld);
    int oa = la ? ntri(la - 1) : 0, ob = lb ? ntri(lb - 1) : 0;
    int oc = lc ? ntri(lc - 1) : 0, od = ld ? ntri(ld - 1) : 0;
    size_t blk = (size_t)ca * cb * cc * cd;
    for (int ij = 0; ij < 6; ++ij) {
        int I = IJ6[ij][0], J = IJ6[ij][1];
        for (int a = 0; a < ca; ++a)
            for (int b = 0; b < cb; ++b) {
                DTerm t0[1] = {{1.0, oa + a, ob + b}}, t1[4], t2[16];
                int n1, n2;
                if (form == 1) {
                    n1 = dterm_apply(t0, 1, t1, J, al, be);
                    n2 = dterm_apply(t1, n1, t2, I, al, be);
                } else {
                    n2 = dterm_apply(t0, 1, t2, I, al, be);
                }
                for (int c = 0; c < cc; ++c)
                    for (int d = 0; d < cd; ++d) {
                        double v = 0.0;
                        if (form == 1) {
                            for (int t = 0; t < n2; ++t)
                                v += t2[t].w * CUM(t2[t].a, t2[t].b, oc + c, od + d);
                        } else {
                            DTerm k0[1] = {{1.0, oc + c, od + d}}, k1[4];
                            int nk = dterm_apply(k0, 1, k1, J, ga, de);
                            for (int t = 0; t < n2; ++t)
                                for (int s = 0; s < nk; ++s)
                                    v -= t2[t].w * k1[s].w * CUM(t2[t].a, t2[t].b, k1[s].a, k1[s].b);
                        }
                        out[ij * blk + ((a * cb + b) * cc + c) * cd + d] = v;
                    }
            }
    }
#undef CUM
    free(cum);
}

/* --------------------------------------------------------- oracle basis */

typedef struct {
    double A[3];
    int nfunc;          /* functions of this shell                        */
    int foff;           /* offset of its first function in its L or S list */
    int nps;            /* primitive shells                                */
    double *alpha;      /* [nps]                                           */
    int *l;             /* [nps]                                           */
    /* sparse map primitive component -> function: for primitive shell s,
       entries [ent_off[s], ent_off[s+1]) of (func, comp, coef)           */
    int *ent_off, *ent_f, *ent_c;
    double *ent_w;
} OrShell;

typedef struct {
    int nL, nS, nsh;      /* nsh = number of L shells (= number of S shells) */
    OrShell *sh;          /* [2 nsh]: L shells then their derivative shells  */
    int *ll;              /* L shell angular momentum                        */
} OrBasis;

static double dfact(int n) { double r = 1.0; for (int k = n; k > 1; k -= 2) r *= k; return r; }

static void shell_alloc_entries(OrShell *s, int nent)
{
    s->ent_f = (int *)malloc(sizeof(int) * (nent > 0 ? nent : 1));
    s->ent_c = (int *)malloc(sizeof(int) * (nent > 0 ? nent : 1));
    s->ent_w = (double *)malloc(sizeof(double) * (nent > 0 ? nent : 1));
}

void *or_basis_create(int n_centers, const double *xyz, int n_shells, const int *shell_center,
                      const int *shell_l, const int *shell_nprim, const double *exps,
                      const double *coefs)
{
    (void)n_centers;
    tri_init();
    OrBasis *B = (OrBasis *)calloc(1, sizeof(OrBasis));
    B->nsh = n_shells;
    B->sh = (OrShell *)calloc(2 * (size_t)n_shells, sizeof(OrShell));
    B->ll = (int *)malloc(sizeof(int) * n_shells);
    int po = 0, fo = 0;
    for (int s = 0; s < n_shells; ++s) {
        int l = shell_l[s], np = shell_nprim[s], nc = ncart(l);
        const double *ex = exps + po, *co = coefs + po;
        B->ll[s] = l;
        /* per-component normalisation: <chi|chi> = 1 */
        double *N = (double *)malloc(sizeof(double) * nc);
        for (int c = 0; c < nc; ++c) {
            int t = (l ? ntri(l - 1) : 0) + c;
            double S = 0.0;
            for (int i = 0; i < np; ++i)
                for (int j = 0; j < np; ++j) {
                    double g = ex[i] + ex[j], v = co[i] * co[j] * pow(M_PI / g, 1.5);
                    for (int d = 0; d < 3; ++d) {
                        int n = g_tri[t][d];
                        v *= dfact(2 * n - 1) / pow(2.0 * g, n);
                    }
                    S += v;
                }
            N[c] = 1.0 / sqrt(S);
        }
        OrShell *L = &B->sh[s], *Sd = &B->sh[n_shells + s];
        for (int d = 0; d < 3; ++d) L->A[d] = Sd->A[d] = xyz[3 * shell_center[s] + d];
        /* large-component shell: primitive shells (alpha_p, l) */
        L->nfunc = nc; L->foff = fo; L->nps = np;
        L->alpha = (double *)malloc(sizeof(double) * np);
        L->l = (int *)malloc(sizeof(int) * np);
        L->ent_off = (int *)malloc(sizeof(int) * (np + 1));
        shell_alloc_entries(L, np * nc);
        int k = 0;
        for (int i = 0; i < np; ++i) {
            L->alpha[i] = ex[i]; L->l[i] = l; L->ent_off[i] = k;
            for (int c = 0; c < nc; ++c) {
                L->ent_f[k] = c; L->ent_c[k] = c; L->ent_w[k] = N[c] * co[i]; ++k;
            }
        }
        L->ent_off[np] = k;
        /* derivative shell: d/dr_K chi_mu = mu_K g_{mu-1_K} - 2 alpha g_{mu+1_K} */
        int nps = l ? 2 * np : np;
        Sd->nfunc = 3 * nc; Sd->foff = 3 * fo; Sd->nps = nps;
        Sd->alpha = (double *)malloc(sizeof(double) * nps);
        Sd->l = (int *)malloc(sizeof(int) * nps);
        Sd->ent_off = (int *)malloc(sizeof(int) * (nps + 1));
        shell_alloc_entries(Sd, nps * 3 * nc);
        k = 0;
        int ps = 0;
        for (int i = 0; i < np; ++i) {
            Sd->alpha[ps] = ex[i]; Sd->l[ps] = l + 1; Sd->ent_off[ps] = k;
            for (int c = 0; c < nc; ++c) {
                int t = (l ? ntri(l - 1) : 0) + c;
                for (int K = 0; K < 3; ++K) {
                    int tp = tri_step(t, K, 1);
                    Sd->ent_f[k] = 3 * c + K; Sd->ent_c[k] = tp - ntri(l);
                    Sd->ent_w[k] = -2.0 * ex[i] * N[c] * co[i]; ++k;
                }
            }
            ++ps;
            if (l) {
                Sd->alpha[ps] = ex[i]; Sd->l[ps] = l - 1; Sd->ent_off[ps] = k;
                for (int c = 0; c < nc; ++c) {
                    int t = ntri(l - 1) + c;
                    for (int K = 0; K < 3; ++K) {
                        if (g_tri[t][K] == 0) continue;
                        int tm = tri_step(t, K, -1);
                        Sd->ent_f[k] = 3 * c + K;
                        Sd->ent_c[k] = tm - (l >= 2 ? ntri(l - 2) : 0);
                        Sd->ent_w[k] = g_tri[t][K] * N[c] * co[i]; ++k;
                    }
                }
                ++ps;
            }
        }
        Sd->ent_off[nps] = k;
        free(N);
        po += np; fo += nc;
    }
    B->nL = fo; B->nS = 3 * fo;
    return B;
}

void or_basis_free(void *h)
{
    OrBasis *B = (OrBasis *)h;
    if (!B) return;
    for (int s = 0; s < 2 * B->nsh; ++s) {
        OrShell *x = &B->sh[s];
        free(x->alpha); free(x->l); free(x->ent_off); free(x->ent_f); free(x->ent_c); free(x->ent_w);
    }
    free(B->sh); free(B->ll); free(B);
}

void or_basis_sizes(void *h, int *out)
{
    OrBasis *B = (OrBasis *)h;
    out[0] = B->nL; out[1] = B->nS; out[2] = B->nsh;
}

/*
 * Contracted block over four oracle shells (index < nsh: L shell, else the
 * derivative shell of L shell index-nsh).
 * mode 0: (ab|1/r12|cd)            out[na][nb][nc][nd]
 * mode 1: (ab|r12|cd)              out[na][nb][nc][nd]
 * mode 2: (ab|K_IJ|cd), K_IJ = r12_I r12_J / r12^3, out[6][na][nb][nc][nd]
 * mode 3: (ab|d_I d_J r12|cd) form 1, mode 4: the same by form 2; out[6][...]
 */
void or_shell_block(void *h, int mode, int sa, int sb, int sc, int sd, double *out)
{
    OrBasis *Bs = (OrBasis *)h;
    const OrShell *S[4] = {&Bs->sh[sa], &Bs->sh[sb], &Bs->sh[sc], &Bs->sh[sd]};
    int na = S[0]->nfunc, nb = S[1]->nfunc, nc = S[2]->nfunc, nd = S[3]->nfunc;
    size_t blk = (size_t)na * nb * nc * nd;
    int ncomp = (mode >= 2) ? 6 : 1;
    memset(out, 0, sizeof(double) * blk * ncomp);
    for (int pa = 0; pa < S[0]->nps; ++pa)
        for (int pb = 0; pb < S[1]->nps; ++pb)
            for (int pc = 0; pc < S[2]->nps; ++pc)
                for (int pd = 0; pd < S[3]->nps; ++pd) {
                    int la = S[0]->l[pa], lb = S[1]->l[pb], lc = S[2]->l[pc], ld = S[3]->l[pd];
                    int ca = ncart(la), cb = ncart(lb), cc = ncart(lc), cd = ncart(ld);
                    size_t pblk = (size_t)ca * cb * cc * cd;
                    double *P = (double *)malloc(sizeof(double) * pblk * 6);
                    if (mode == 0 || mode == 1) {
                        or_prim_block(mode, S[0]->A, S[0]->alpha[pa], la, S[1]->A, S[1]->alpha[pb], lb,
                                      S[2]->A, S[2]->alpha[pc], lc, S[3]->A, S[3]->alpha[pd], ld, P);
                    } else {
                        or_prim_ddr(mode == 4 ? 2 : 1, S[0]->A, S[0]->alpha[pa], la, S[1]->A,
                                    S[1]->alpha[pb], lb, S[2]->A, S[2]->alpha[pc], lc, S[3]->A,
                                    S[3]->alpha[pd], ld, P);
                        if (mode == 2) {
                            /* K_IJ = delta_IJ / r12 - d_I d_J r12 */
                            double *Cb = (double *)malloc(sizeof(double) * pblk);
                            or_prim_block(0, S[0]->A, S[0]->alpha[pa], la, S[1]->A, S[1]->alpha[pb], lb,
                                          S[2]->A, S[2]->alpha[pc], lc, S[3]->A, S[3]->alpha[pd], ld, Cb);
                            for (int ij = 0; ij < 6; ++ij) {
                                double diag = (IJ6[ij][0] == IJ6[ij][1]) ? 1.0 : 0.0;
                                for (size_t x = 0; x < pblk; ++x)
                                    P[ij * pblk + x] = diag * Cb[x] - P[ij * pblk + x];
                            }
                            free(Cb);
                        }
                    }
                    for (int ea = S[0]->ent_off[pa]; ea < S[0]->ent_off[pa + 1]; ++ea)
                        for (int eb = S[1]->ent_off[pb]; eb < S[1]->ent_off[pb + 1]; ++eb)
                            for (int ec = S[2]->ent_off[pc]; ec < S[2]->ent_off[pc + 1]; ++ec)
                                for (int ed = S[3]->ent_off[pd]; ed < S[3]->ent_off[pd + 1]; ++ed) {
                                    double w = S[0]->ent_w[ea] * S[1]->ent_w[eb] * S[2]->ent_w[ec] *
                                               S[3]->ent_w[ed];
                                    size_t po = ((size_t)(S[0]->ent_c[ea] * cb + S[1]->ent_c[eb]) * cc +
                                                 S[2]->ent_c[ec]) * cd + S[3]->ent_c[ed];
                                    size_t fo = ((size_t)(S[0]->ent_f[ea] * nb + S[1]->ent_f[eb]) * nc +
                                                 S[2]->ent_f[ec]) * nd + S[3]->ent_f[ed];
                                    for (int k = 0; k < ncomp; ++k)
                                        out[k * blk + fo] += w * P[k * pblk + po];
                                }
                    free(P);
                }
}

/* ---------------------------------------------------- pair matrices */

/*
 * Function-pair orders used by the oracle:
 *   class 0 (Coulomb): LL pairs a<=b (row-major over a), then SS pairs a<=b;
 *   class 1 (LS, Gaunt and gauge): (a in L, b in S), index a*nS + b.
 * Shell pairs: class 0 = LL shell pairs A<=B then SS shell pairs A<=B;
 *              class 1 = (A in L shells, B in S shells).
 */
static long pair_tri(long a, long b, long n) { return a * n - a * (a - 1) / 2 + (b - a); }

typedef struct { int sa, sb; } SPair;

static int shell_pairs(const OrBasis *B, int cls, SPair **out)
{
    int n = B->nsh, k = 0;
    int cnt = cls == 0 ? n * (n + 1) : n * n;
    SPair *p = (SPair *)malloc(sizeof(SPair) * cnt);
    if (cls == 0) {
        for (int off = 0; off <= n; off += n)
            for (int a = 0; a < n; ++a)
                for (int b = a; b < n; ++b) p[k++] = (SPair){a + off, b + off};
    } else {
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) p[k++] = (SPair){a, b + n};
    }
    *out = p;
    return k;
}

/* global pair index of function pair (fa, fb) of shells (sa, sb); -1 if not stored */
static long pair_index(const OrBasis *B, int cls, int sa, int sb, int fa, int fb)
{
    int n = B->nsh;
    if (cls == 0) {
        int isS = sa >= n;
        long a = (isS ? B->sh[sa].foff : B->sh[sa].foff) + fa;
        long b = (isS ? B->sh[sb].foff : B->sh[sb].foff) + fb;
        if (a > b) return -1;
        long NL = B->nL;
        if (!isS) return pair_tri(a, b, NL);
        return NL * (NL + 1) / 2 + pair_tri(a, b, B->nS);
    }
    long a = B->sh[sa].foff + fa, b = B->sh[sb].foff + fb;
    return a * B->nS + b;
}

long or_npairs(void *h, int cls)
{
    OrBasis *B = (OrBasis *)h;
    long NL = B->nL, NS = B->nS;
    return cls == 0 ? NL * (NL + 1) / 2 + NS * (NS + 1) / 2 : NL * NS;
}

/*
 * Rows of a pair matrix:
 *   cls 0, kernel 0: G_C[row][col] = (ab|cd), col over all class-0 pairs
 *   cls 1, kernel 0: G_G[row][col] = (ab|cd) over LS pairs
 *   cls 1, kernel 2: [row][6][col] = (ab|K_IJ|cd) over LS pairs
 * rows: nrows global pair indices of the class; out is zero-filled first.
 */
void or_pair_rows(void *h, int cls, int kernel, long nrows, const long *rows, double *out)
{
    OrBasis *B = (OrBasis *)h;
    SPair *sp;
    int nsp = shell_pairs(B, cls, &sp);
    long M = or_npairs(h, cls);
    int ncomp = kernel == 2 ? 6 : 1;
    memset(out, 0, sizeof(double) * (size_t)nrows * ncomp * M);
    /* which bra shell pairs are needed */
    char *need = (char *)calloc(nsp, 1);
    for (int p = 0; p < nsp; ++p) {
        const OrShell *A = &B->sh[sp[p].sa], *Bb = &B->sh[sp[p].sb];
        for (int fa = 0; fa < A->nfunc; ++fa)
            for (int fb = 0; fb < Bb->nfunc; ++fb) {
                long g = pair_index(B, cls, sp[p].sa, sp[p].sb, fa, fb);
                if (g < 0) continue;
                for (long r = 0; r < nrows; ++r)
                    if (rows[r] == g) need[p] = 1;
            }
    }
    for (int p = 0; p < nsp; ++p) {
        if (!need[p]) continue;
        const OrShell *A = &B->sh[sp[p].sa], *Bb = &B->sh[sp[p].sb];
#pragma omp parallel for schedule(dynamic)
        for (int q = 0; q < nsp; ++q) {
            const OrShell *Cc = &B->sh[sp[q].sa], *Dd = &B->sh[sp[q].sb];
            int na = A->nfunc, nb = Bb->nfunc, nc = Cc->nfunc, nd = Dd->nfunc;
            size_t blk = (size_t)na * nb * nc * nd;
            double *buf = (double *)malloc(sizeof(double) * blk * ncomp);
            int mode = kernel == 2 ? 2 : 0;
            or_shell_block(h, mode, sp[p].sa, sp[p].sb, sp[q].sa, sp[q].sb, buf);
            for (int fa = 0; fa < na; ++fa)
                for (int fb = 0; fb < nb; ++fb) {
                    long g = pair_index(B, cls, sp[p].sa, sp[p].sb, fa, fb);
                    if (g < 0) continue;
                    for (long r = 0; r < nrows; ++r) {
                        if (rows[r] != g) continue;
                        for (int fc = 0; fc < nc; ++fc)
                            for (int fd = 0; fd < nd; ++fd) {
                                long col = pair_index(B, cls, sp[q].sa, sp[q].sb, fc, fd);
                                if (col < 0) continue;
                                for (int k = 0; k < ncomp; ++k)
                                    out[((size_t)r * ncomp + k) * M + col] =
                                        buf[k * blk + ((size_t)(fa * nb + fb) * nc + fc) * nd + fd];
                            }
                    }
                }
            free(buf);
        }
    }
    free(need); free(sp);
}

/*
 * Row-streamed form of the pair matrix for one bra shell pair p of a class:
 * the rows of its stored function pairs (fa major, fb minor), computed only
 * against the ket shell pairs q with keep[q] != 0 -- the shell quartets that
 * the screening of Eq. SchwarzDen keeps; the columns of the other ket shell
 * pairs stay zero.  rows_out[r] receives the global pair index of row r,
 * out[r][k][col] the value (k < 6 components for kernel 2, else 1); out holds
 * nfunc_A * nfunc_B * ncomp * M doubles.  Returns the number of rows.
 */
long or_shell_pair_rows(void *h, int cls, int kernel, int p, const unsigned char *keep, long *rows_out,
                        double *out)
{
    OrBasis *B = (OrBasis *)h;
    SPair *sp;
    int nsp = shell_pairs(B, cls, &sp);
    long M = or_npairs(h, cls);
    int ncomp = kernel == 2 ? 6 : 1;
    const OrShell *A = &B->sh[sp[p].sa], *Bb = &B->sh[sp[p].sb];
    int na = A->nfunc, nb = Bb->nfunc;
    int *rl = (int *)malloc(sizeof(int) * na * nb);
    long nrows = 0;
    for (int fa = 0; fa < na; ++fa)
        for (int fb = 0; fb < nb; ++fb) {
            long g = pair_index(B, cls, sp[p].sa, sp[p].sb, fa, fb);
            rl[fa * nb + fb] = g < 0 ? -1 : (int)nrows;
            if (g >= 0) rows_out[nrows++] = g;
        }
    memset(out, 0, sizeof(double) * (size_t)nrows * ncomp * M);
#pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < nsp; ++q) {
        if (!keep[q]) continue;
        const OrShell *Cc = &B->sh[sp[q].sa], *Dd = &B->sh[sp[q].sb];
        int nc = Cc->nfunc, nd = Dd->nfunc;
        size_t blk = (size_t)na * nb * nc * nd;
        double *buf = (double *)malloc(sizeof(double) * blk * ncomp);
        or_shell_block(h, kernel == 2 ? 2 : 0, sp[p].sa, sp[p].sb, sp[q].sa, sp[q].sb, buf);
        for (int fa = 0; fa < na; ++fa)
            for (int fb = 0; fb < nb; ++fb) {
                int r = rl[fa * nb + fb];
                if (r < 0) continue;
                for (int fc = 0; fc < nc; ++fc)
                    for (int fd = 0; fd < nd; ++fd) {
                        long col = pair_index(B, cls, sp[q].sa, sp[q].sb, fc, fd);
                        if (col < 0) continue;
                        for (int k = 0; k < ncomp; ++k)
                            out[((size_t)r * ncomp + k) * M + col] =
                                buf[k * blk + ((size_t)(fa * nb + fb) * nc + fc) * nd + fd];
                    }
            }
        free(buf);
    }
    free(rl); free(sp);
    return nrows;
}

/* Full pair matrix: cls 0 -> [M][M]; cls 1 kernel 0 -> [M][M];
   cls 1 kernel 2 -> [6][M][M] (note the component-major layout). */
void or_pair_matrix(void *h, int cls, int kernel, double *out)
{
    OrBasis *B = (OrBasis *)h;
    SPair *sp;
    int nsp = shell_pairs(B, cls, &sp);
    long M = or_npairs(h, cls);
    int ncomp = kernel == 2 ? 6 : 1;
    memset(out, 0, sizeof(double) * (size_t)ncomp * M * M);
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int p = 0; p < nsp; ++p)
        for (int q = 0; q < nsp; ++q) {
            if (q < p) continue;
            const OrShell *A = &B->sh[sp[p].sa], *Bb = &B->sh[sp[p].sb];
            const OrShell *Cc = &B->sh[sp[q].sa], *Dd = &B->sh[sp[q].sb];
            int na = A->nfunc, nb = Bb->nfunc, nc = Cc->nfunc, nd = Dd->nfunc;
            size_t blk = (size_t)na * nb * nc * nd;
            double *buf = (double *)malloc(sizeof(double) * blk * ncomp);
            or_shell_block(h, kernel == 2 ? 2 : 0, sp[p].sa, sp[p].sb, sp[q].sa, sp[q].sb, buf);
            for (int fa = 0; fa < na; ++fa)
                for (int fb = 0; fb < nb; ++fb) {
                    long r = pair_index(B, cls, sp[p].sa, sp[p].sb, fa, fb);
                    if (r < 0) continue;
                    for (int fc = 0; fc < nc; ++fc)
                        for (int fd = 0; fd < nd; ++fd) {
                            long c = pair_index(B, cls, sp[q].sa, sp[q].sb, fc, fd);
                            if (c < 0) continue;
                            for (int k = 0; k < ncomp; ++k) {
                                double v = buf[k * blk + ((size_t)(fa * nb + fb) * nc + fc) * nd + fd];
                                out[((size_t)k * M + r) * M + c] = v;   /* (ab|K_IJ|cd) */
                                out[((size_t)k * M + c) * M + r] = v;   /* = (cd|K_JI|ab), K symmetric */
                            }
                        }
                }
            free(buf);
        }
    free(sp);
}

/* Diagonal (ab|ab) of the Coulomb pair matrix of a class. */
void or_pair_diag(void *h, int cls, double *out)
{
    OrBasis *B = (OrBasis *)h;
    SPair *sp;
    int nsp = shell_pairs(B, cls, &sp);
#pragma omp parallel for schedule(dynamic)
    for (int p = 0; p < nsp; ++p) {
        const OrShell *A = &B->sh[sp[p].sa], *Bb = &B->sh[sp[p].sb];
        int na = A->nfunc, nb = Bb->nfunc;
        double *buf = (double *)malloc(sizeof(double) * (size_t)na * nb * na * nb);
        or_shell_block(h, 0, sp[p].sa, sp[p].sb, sp[p].sa, sp[p].sb, buf);
        for (int fa = 0; fa < na; ++fa)
            for (int fb = 0; fb < nb; ++fb) {
                long g = pair_index(B, cls, sp[p].sa, sp[p].sb, fa, fb);
                if (g < 0) continue;
                out[g] = buf[((size_t)(fa * nb + fb) * na + fa) * nb + fb];
            }
        free(buf);
    }
    free(sp);
}

/* ------------------------------------------------------------- overlaps */

/* 1D overlap table S[i][j] = int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) dx
   by the Obara-Saika recursion; i <= li, j <= lj. */
static void overlap_1d(double A, double a, int li, double B, double b, int lj, double *S)
{
    double p = a + b, P = (a * A + b * B) / p, PA = P - A, PB = P - B;
    int n = lj + 1;
    for (int i = 0; i <= li; ++i)
        for (int j = 0; j <= lj; ++j) S[i * n + j] = 0.0;
    S[0] = sqrt(M_PI / p) * exp(-a * b / p * (A - B) * (A - B));
    for (int i = 0; i <= li; ++i)
        for (int j = 0; j <= lj; ++j) {
            if (i == 0 && j == 0) continue;
            double v;
            if (i > 0) {
                v = PA * S[(i - 1) * n + j];
                if (i > 1) v += (i - 1) / (2.0 * p) * S[(i - 2) * n + j];
                if (j > 0) v += j / (2.0 * p) * S[(i - 1) * n + j - 1];
            } else {
                v = PB * S[j - 1];
                if (j > 1) v += (j - 1) / (2.0 * p) * S[j - 2];
            }
            S[i * n + j] = v;
        }
}

/* Overlap block <chi_a | chi_b> over two oracle shells: out[na][nb]. */
void or_overlap_block(void *h, int sa, int sb, double *out)
{
    OrBasis *Bs = (OrBasis *)h;
    const OrShell *X = &Bs->sh[sa], *Y = &Bs->sh[sb];
    int na = X->nfunc, nb = Y->nfunc;
    memset(out, 0, sizeof(double) * na * nb);
    double S[3][16 * 16];
    for (int pa = 0; pa < X->nps; ++pa)
        for (int pb = 0; pb < Y->nps; ++pb) {
            int la = X->l[pa], lb = Y->l[pb];
            for (int d = 0; d < 3; ++d)
                overlap_1d(X->A[d], X->alpha[pa], la, Y->A[d], Y->alpha[pb], lb, S[d]);
            for (int ea = X->ent_off[pa]; ea < X->ent_off[pa + 1]; ++ea)
                for (int eb = Y->ent_off[pb]; eb < Y->ent_off[pb + 1]; ++eb) {
                    int ta = (la ? ntri(la - 1) : 0) + X->ent_c[ea];
                    int tb = (lb ? ntri(lb - 1) : 0) + Y->ent_c[eb];
                    double v = X->ent_w[ea] * Y->ent_w[eb];
                    for (int d = 0; d < 3; ++d) v *= S[d][g_tri[ta][d] * (lb + 1) + g_tri[tb][d]];
                    out[X->ent_f[ea] * nb + Y->ent_f[eb]] += v;
                }
        }
}

/* Threads of the OpenMP loops above (timing on a given number of host cores). */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
