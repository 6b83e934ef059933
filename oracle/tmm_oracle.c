/*
 * tmm_oracle.c -- the oracle: a plain, slow FP64 CPU implementation of the
 * coherent transfer-matrix method (Abeles) of TMM-Fast, arXiv 2111.13667.
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by the test-suite, by the smoke
 * check and by the benchmark's CPU-baseline leg, and by nothing else.  It
 * shares no code, header, table or helper with the CUDA path; the product
 * library never links or calls it.
 *
 * What it computes, step by step in the paper's order (Sec. 2):
 *   1. Snell's law (Sec. 2, first paragraph): with the incidence angle theta
 *      given in the injection medium 0, beta = n_0 sin(theta) is invariant
 *      and cos(theta_j) = sqrt(1 - (beta / n_j)^2) in every medium j.
 *      The paper does not say which square root to take.  Reading used here:
 *      the root for which n_j cos(theta_j) has a positive imaginary part (a
 *      wave that decays along +z); when that imaginary part is zero up to
 *      rounding (|Im| <= 100 eps |n c|), the root with positive real part
 *      (a wave that propagates along +z).
 *   2. Fresnel coefficients, Eq. 1, with mu_r = 1, for every interface
 *      j -> j+1 and the requested polarisation, exactly as printed:
 *        s: r = (n1 c1 - n2 c2) / (n1 c1 + n2 c2),  t = 2 n1 c1 / (n1 c1 + n2 c2)
 *        p: r = (n2 c1 - n1 c2) / (n2 c1 + n1 c2),  t = 2 n1 c1 / (n2 c1 + n1 c2)
 *   3. Phase of each finite layer (text after Eq. 3): delta_j = d_j k_z =
 *      2 pi n_j d_j cos(theta_j) / lambda.  Opaque-layer clamp (not in the
 *      paper; a reading): Im(delta_j) is limited to 35, which changes R and T
 *      by a relative O(exp(-35)) and keeps the product finite.
 *   4. Layer matrices, Eq. 3: M_j = diag(e^{-i delta_j}, e^{i delta_j})
 *      [[1, r_j],[r_j, 1]] / t_j, where r_j, t_j belong to the interface
 *      j -> j+1.  The semi-infinite medium 0 carries no phase, so its matrix
 *      is [[1, r_0],[r_0, 1]] / t_0.
 *   5. Characteristic matrix, Eq. 4: M~ = M_0 M_1 ... M_L, multiplied as full
 *      2x2 complex matrices from left to right.
 *   6. Eqs. 5-6: (1, r)^T = M~ (t, 0)^T, so r = M~_10 / M~_00, t = 1 / M~_00.
 *   7. Eq. 2 (garbled in the paper; read as the Poynting-flux form):
 *        R = |r|^2
 *        s: T = Re(n_out c_out) / Re(n_in c_in) |t|^2
 *        p: T = Re(n_out conj(c_out)) / Re(n_in conj(c_in)) |t|^2
 *      At exact grazing incidence (cos(theta_0) = 0) the ratio is 0/0; the
 *      reading used is R = 1, T = 0.
 *
 * The gradient entry point differentiates the per-stack merit
 *   m_s = mean over (lambda, theta, pol) of (R - R_target)^2
 * (the mean-squared-error merit of the paper's Sec. 4 / appendix example)
 * with respect to every thickness d_j and a real offset Delta n_j added to
 * the index of layer j at every wavelength.  It uses forward-mode dual
 * numbers (value, derivative) pushed through the very same steps 1-7, one
 * parameter at a time.  No reverse sweep is involved.
 *
 * Arrays are plain host memory, C order.  Complex arrays are interleaved
 * (re, im) doubles.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_IM_DELTA_MAX 35.0

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Step 1: Snell's law and the root choice.                                   */
/* ------------------------------------------------------------------------- */
static cplx cos_theta_in(cplx n, double beta, int flip)
{
    cplx s = beta / n;
    cplx c = csqrt(1.0 - s * s);
    cplx nc = n * c;
    if (fabs(cimag(nc)) <= 100.0 * DBL_EPSILON * cabs(nc)) {
        if (creal(nc) < 0.0) c = -c;
    } else if (cimag(nc) < 0.0) {
        c = -c;
    }
    /* Test hook only: take the other root in an interior layer. */
    if (flip) c = -c;
    return c;
}

/* Step 2: Eq. 1 with mu_r = 1.  pol 0 = s, 1 = p. */
static void fresnel(int pol, cplx n1, cplx n2, cplx c1, cplx c2, cplx *r, cplx *t)
{
    if (pol == 0) {
        cplx den = n1 * c1 + n2 * c2;
        *r = (n1 * c1 - n2 * c2) / den;
        *t = 2.0 * n1 * c1 / den;
    } else {
        cplx den = n2 * c1 + n1 * c2;
        *r = (n2 * c1 - n1 * c2) / den;
        *t = 2.0 * n1 * c1 / den;
    }
}

typedef struct { cplx a, b, c, d; } mat2; /* [[a, b], [c, d]] */

static mat2 mat2_mul(mat2 x, mat2 y)
{
    mat2 z;
    z.a = x.a * y.a + x.b * y.c;
    z.b = x.a * y.b + x.b * y.d;
    z.c = x.c * y.a + x.d * y.c;
    z.d = x.c * y.b + x.d * y.d;
    return z;
}

/*
 * One (stack, theta, lambda, pol) evaluation.  n points at the stack's row of
 * media (index 0 = injection medium, L+1 = outcoupling medium, stride nstride
 * doubles-complex between media), d at its L finite thicknesses.
 */
static void tmm_one(int pol, int L, const cplx *n, long nstride, const double *d,
                    double theta, double lambda, uint32_t flip_mask,
                    double *R_out, double *T_out)
{
    cplx *c = (cplx *)malloc(sizeof(cplx) * (size_t)(L + 2));
    const double beta = creal(n[0]) * sin(theta);
    for (int j = 0; j <= L + 1; ++j) {
        int flip = (j >= 1 && j <= L && j <= 32) ? (int)((flip_mask >> (j - 1)) & 1u) : 0;
        c[j] = cos_theta_in(n[(long)j * nstride], beta, flip);
    }
    if (c[0] == 0.0) { /* exact grazing incidence */
        *R_out = 1.0;
        *T_out = 0.0;
        free(c);
        return;
    }
    cplx r0, t0;
    fresnel(pol, n[0], n[nstride], c[0], c[1], &r0, &t0);
    mat2 M = {1.0 / t0, r0 / t0, r0 / t0, 1.0 / t0};
    for (int j = 1; j <= L; ++j) {
        cplx nj = n[(long)j * nstride];
        cplx rj, tj;
        fresnel(pol, nj, n[(long)(j + 1) * nstride], c[j], c[j + 1], &rj, &tj);
        cplx delta = 2.0 * M_PI * nj * d[j - 1] * c[j] / lambda;
        if (cimag(delta) > ORACLE_IM_DELTA_MAX) delta = creal(delta) + I * ORACLE_IM_DELTA_MAX;
        cplx em = cexp(-I * delta), ep = cexp(I * delta);
        mat2 Mj = {em / tj, em * rj / tj, ep * rj / tj, ep / tj};
        M = mat2_mul(M, Mj);
    }
    cplx r = M.c / M.a;
    cplx t = 1.0 / M.a;
    cplx nin = n[0], nout = n[(long)(L + 1) * nstride];
    double R = creal(r * conj(r));
    double T;
    if (pol == 0)
        T = creal(nout * c[L + 1]) / creal(nin * c[0]) * creal(t * conj(t));
    else
        T = creal(nout * conj(c[L + 1])) / creal(nin * conj(c[0])) * creal(t * conj(t));
    *R_out = R;
    *T_out = T;
    free(c);
}

/* ------------------------------------------------------------------------- */
/* Threading: a shared item counter, one worker per host thread.             */
/* ------------------------------------------------------------------------- */
typedef struct {
    int pol, S, L_max, Nl, Nt;
    const cplx *n;
    const double *d;
    const int32_t *L_per_stack;
    const double *theta, *lambda;
    const uint32_t *flip_mask;
    double *R, *T;
    long n_items;
    long next;
} fwd_job;

static void *fwd_worker(void *arg)
{
    fwd_job *jb = (fwd_job *)arg;
    const long per_stack_media = (long)(jb->L_max + 2) * jb->Nl;
    for (;;) {
        long it = __atomic_fetch_add(&jb->next, 1, __ATOMIC_RELAXED);
        if (it >= jb->n_items) break;
        int s = (int)(it / jb->Nt), a = (int)(it % jb->Nt);
        int L = jb->L_per_stack ? jb->L_per_stack[s] : jb->L_max;
        uint32_t fm = jb->flip_mask ? jb->flip_mask[s] : 0u;
        for (int l = 0; l < jb->Nl; ++l) {
            long o = ((long)s * jb->Nt + a) * jb->Nl + l;
            tmm_one(jb->pol, L, jb->n + (long)s * per_stack_media + l, jb->Nl,
                    jb->d + (long)s * jb->L_max, jb->theta[a], jb->lambda[l], fm,
                    &jb->R[o], &jb->T[o]);
        }
    }
    return NULL;
}

static void run_workers(void *(*fn)(void *), void *job, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads == 1) {
        fn(job);
        return;
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int started = 0;
    for (int i = 0; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, fn, job) == 0) ++started;
    if (started == 0) fn(job);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    free(th);
}

/*
 * R, T for one polarisation over every (stack, theta, lambda).
 *   pol          0 = s, 1 = p
 *   n            complex [S][L_max+2][Nl]: media 0..L_s+1 of each stack; for a
 *                stack with L_s < L_max, entry L_s+1 is its outcoupling medium
 *   d            [S][L_max] thicknesses in nm (entries past L_s ignored)
 *   L_per_stack  [S] finite-layer count of each stack, or NULL (= L_max)
 *   theta        [Nt] angle of incidence in medium 0, radians
 *   lambda       [Nl] vacuum wavelength, nm
 *   flip_mask    [S] or NULL; test hook: bit j-1 takes the other root of
 *                cos(theta_j) in interior layer j (j <= 32)
 *   R, T         [S][Nt][Nl] outputs
 * Returns 0, or -1 on a bad argument.
 */
int oracle_coh_tmm(int pol, int S, int L_max, int Nl, int Nt, const double *n,
                   const double *d, const int32_t *L_per_stack, const double *theta,
                   const double *lambda, const uint32_t *flip_mask, double *R,
                   double *T, int nthreads)
{
    if ((pol != 0 && pol != 1) || S < 0 || L_max < 0 || Nl < 0 || Nt < 0) return -1;
    if (L_per_stack)
        for (int s = 0; s < S; ++s)
            if (L_per_stack[s] < 0 || L_per_stack[s] > L_max) return -1;
    fwd_job jb = {pol, S, L_max, Nl, Nt, (const cplx *)n, d, L_per_stack, theta, lambda,
                  flip_mask, R, T, (long)S * Nt, 0};
    run_workers(fwd_worker, &jb, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Forward-mode dual numbers for the gradient.                                */
/* ------------------------------------------------------------------------- */
typedef struct { cplx v, e; } dual; /* value and derivative wrt one parameter */

static dual dl(cplx v) { dual r = {v, 0.0}; return r; }
static dual dadd(dual a, dual b) { dual r = {a.v + b.v, a.e + b.e}; return r; }
static dual dsub(dual a, dual b) { dual r = {a.v - b.v, a.e - b.e}; return r; }
static dual dmul(dual a, dual b) { dual r = {a.v * b.v, a.e * b.v + a.v * b.e}; return r; }
static dual dscale(cplx k, dual a) { dual r = {k * a.v, k * a.e}; return r; }
static dual ddiv(dual a, dual b)
{
    cplx q = a.v / b.v;
    dual r = {q, (a.e - q * b.e) / b.v};
    return r;
}
static dual dexp(dual a)
{
    cplx ev = cexp(a.v);
    dual r = {ev, ev * a.e};
    return r;
}

/* Step 1 in duals: c^2 = 1 - beta^2 / n^2, so dc = beta^2 dn / (n^3 c). */
static dual dcos_theta_in(dual n, double beta)
{
    cplx c = cos_theta_in(n.v, beta, 0);
    dual r = {c, 0.0};
    if (n.e != 0.0) r.e = beta * beta * n.e / (n.v * n.v * n.v * c);
    return r;
}

static void dfresnel(int pol, dual n1, dual n2, dual c1, dual c2, dual *r, dual *t)
{
    dual two = dl(2.0);
    if (pol == 0) {
        dual a = dmul(n1, c1), b = dmul(n2, c2);
        dual den = dadd(a, b);
        *r = ddiv(dsub(a, b), den);
        *t = ddiv(dmul(two, a), den);
    } else {
        dual a = dmul(n2, c1), b = dmul(n1, c2);
        dual den = dadd(a, b);
        *r = ddiv(dsub(a, b), den);
        *t = ddiv(dmul(two, dmul(n1, c1)), den);
    }
}

typedef struct { dual a, b, c, d; } dmat2;

static dmat2 dmat2_mul(dmat2 x, dmat2 y)
{
    dmat2 z;
    z.a = dadd(dmul(x.a, y.a), dmul(x.b, y.c));
    z.b = dadd(dmul(x.a, y.b), dmul(x.b, y.d));
    z.c = dadd(dmul(x.c, y.a), dmul(x.d, y.c));
    z.d = dadd(dmul(x.c, y.b), dmul(x.d, y.d));
    return z;
}

/*
 * R and dR/dp for one (stack, theta, lambda, pol); the parameter p is the
 * thickness of layer jp (kind 0) or a real offset of its index (kind 1);
 * jp = 0 means "no parameter" (derivative 0).
 */
static void tmm_one_dual(int pol, int L, const cplx *n, long nstride, const double *d,
                         double theta, double lambda, int kind, int jp, double *R_out,
                         double *dR_out)
{
    dual *nn = (dual *)malloc(sizeof(dual) * (size_t)(L + 2));
    dual *c = (dual *)malloc(sizeof(dual) * (size_t)(L + 2));
    const double beta = creal(n[0]) * sin(theta);
    for (int j = 0; j <= L + 1; ++j) {
        nn[j] = dl(n[(long)j * nstride]);
        if (kind == 1 && j == jp) nn[j].e = 1.0;
        c[j] = dcos_theta_in(nn[j], beta);
    }
    if (c[0].v == 0.0) {
        *R_out = 1.0;
        *dR_out = 0.0;
        free(nn);
        free(c);
        return;
    }
    dual r0, t0;
    dfresnel(pol, nn[0], nn[1], c[0], c[1], &r0, &t0);
    dual one = dl(1.0);
    dmat2 M = {ddiv(one, t0), ddiv(r0, t0), ddiv(r0, t0), ddiv(one, t0)};
    for (int j = 1; j <= L; ++j) {
        dual rj, tj;
        dfresnel(pol, nn[j], nn[j + 1], c[j], c[j + 1], &rj, &tj);
        dual dj = dl(d[j - 1]);
        if (kind == 0 && j == jp) dj.e = 1.0;
        dual delta = dscale(2.0 * M_PI / lambda, dmul(dmul(nn[j], dj), c[j]));
        if (cimag(delta.v) > ORACLE_IM_DELTA_MAX) {
            delta.v = creal(delta.v) + I * ORACLE_IM_DELTA_MAX;
            delta.e = creal(delta.e); /* the clamped imaginary part is constant */
        }
        dual em = dexp(dscale(-I, delta)), ep = dexp(dscale(I, delta));
        dmat2 Mj = {ddiv(em, tj), ddiv(dmul(em, rj), tj), ddiv(dmul(ep, rj), tj), ddiv(ep, tj)};
        M = dmat2_mul(M, Mj);
    }
    dual r = ddiv(M.c, M.a);
    *R_out = creal(r.v * conj(r.v));
    *dR_out = 2.0 * creal(conj(r.v) * r.e);
    free(nn);
    free(c);
}

typedef struct {
    int pol_mask, S, L_max, Nl, Nt;
    const cplx *n;
    const double *d;
    const int32_t *L_per_stack;
    const double *theta, *lambda, *R_target;
    double *merit, *dm_dd, *dm_dn;
    long n_items;
    long next;
} grad_job;

static void *grad_worker(void *arg)
{
    grad_job *jb = (grad_job *)arg;
    const long per_stack_media = (long)(jb->L_max + 2) * jb->Nl;
    const int per = 1 + 2 * jb->L_max;
    int npol = ((jb->pol_mask & 1u) ? 1 : 0) + ((jb->pol_mask & 2u) ? 1 : 0);
    const double norm = 1.0 / ((double)npol * jb->Nt * jb->Nl);
    for (;;) {
        long it = __atomic_fetch_add(&jb->next, 1, __ATOMIC_RELAXED);
        if (it >= jb->n_items) break;
        int s = (int)(it / per), q = (int)(it % per);
        int L = jb->L_per_stack ? jb->L_per_stack[s] : jb->L_max;
        int kind = 0, jp = 0;
        if (q >= 1 && q <= jb->L_max) { kind = 0; jp = q; }
        if (q > jb->L_max) { kind = 1; jp = q - jb->L_max; }
        double *dst = q == 0 ? &jb->merit[s]
                    : kind == 0 ? &jb->dm_dd[(long)s * jb->L_max + jp - 1]
                                : &jb->dm_dn[(long)s * jb->L_max + jp - 1];
        if (jp > L) { *dst = 0.0; continue; }
        double acc = 0.0;
        int pi = 0;
        for (int pol = 0; pol < 2; ++pol) {
            if (!((jb->pol_mask >> pol) & 1u)) continue;
            for (int a = 0; a < jb->Nt; ++a)
                for (int l = 0; l < jb->Nl; ++l) {
                    double R, dR;
                    tmm_one_dual(pol, L, jb->n + (long)s * per_stack_media + l, jb->Nl,
                                 jb->d + (long)s * jb->L_max, jb->theta[a], jb->lambda[l],
                                 kind, jp, &R, &dR);
                    double e = R - jb->R_target[((long)pi * jb->Nt + a) * jb->Nl + l];
                    acc += q == 0 ? e * e : 2.0 * e * dR;
                }
            ++pi;
        }
        *dst = acc * norm;
    }
    return NULL;
}

/*
 * Merit m_s = mean over (pol, theta, lambda) of (R - R_target)^2 per stack,
 * and its derivatives with respect to every d_j (dm_dd, 1/nm) and a real
 * offset of n_j (dm_dn), j = 1..L_s; entries past L_s are written as 0.
 *   pol_mask     bit 0 = s, bit 1 = p (at least one)
 *   R_target     [P][Nt][Nl], P = number of bits set, s before p
 *   merit        [S]; dm_dd, dm_dn: [S][L_max]
 * Other arguments as for oracle_coh_tmm.  Returns 0, or -1 on a bad argument.
 */
int oracle_merit_grad(int pol_mask, int S, int L_max, int Nl, int Nt, const double *n,
                      const double *d, const int32_t *L_per_stack, const double *theta,
                      const double *lambda, const double *R_target, double *merit,
                      double *dm_dd, double *dm_dn, int nthreads)
{
    if ((pol_mask & 3) == 0 || (pol_mask & ~3) || S < 0 || L_max < 0 || Nl <= 0 || Nt <= 0)
        return -1;
    grad_job jb = {pol_mask, S, L_max, Nl, Nt, (const cplx *)n, d, L_per_stack,
                   theta, lambda, R_target, merit, dm_dd, dm_dn,
                   (long)S * (1 + 2 * L_max), 0};
    run_workers(grad_worker, &jb, nthreads);
    return 0;
}
