/*
 * mpbp_oracle.c -- plain FP64 CPU oracle for the multi-peak Bragg
 * ptychography (MPBP) loss and gradient (Kandel et al., arXiv 2312.14907).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product library never does.
 * It shares no code, header, table or helper with the CUDA sources.
 *
 * What it computes, in the paper's notation (thin-membrane form, R = identity):
 *   Eq. 1 / Eq. 3   O_m(r)   = alpha_m rho(r) exp(i phi_m(r)),
 *                   phi_m(r) = phase_scale * sum_c G_{m,c} u_c(r)
 *                   (phase_scale = 2 pi reproduces the exponent 2 pi i u.G).
 *   Eq. 2           I_{m,j}  = | F diag(P_m) S_j O_m |^2 + b_{m,j}
 *                   S_j: integer shift, z(k) = O_m(s_j + k), zero outside the
 *                   grid; F: unnormalised 2-D DFT with kernel exp(-2 pi i q.k/M),
 *                   evaluated here as a direct separable sum (no FFT).
 *   Eq. 4           f = 1/2 sum_{m,j,q} ( sqrt(I) - sqrt(y) )^2
 *   gradient of Eq. 4 with respect to rho, u and alpha (what Alg. 1 feeds its
 *   optimizer), by the chain rule through Eq. 2 and Eq. 3:
 *     chi  = (sqrt(I) - sqrt(y)) Psi / sqrt(I)      (chi = 0 where I = 0)
 *     ghat = F^H chi                                (conjugate transpose DFT)
 *     g    = conj(P) ghat
 *     df/drho(r)   += alpha_m Re( conj(g) e^{i phi_m(r)} )
 *     df/dphi_m(r) += -Im( conj(g) O_m(r) )
 *     df/dalpha_m  += Re( conj(g) rho(r) e^{i phi_m(r)} )
 *     df/du_c(r)    = phase_scale * sum_m G_{m,c} df/dphi_m(r)
 *
 * Also: the per-peak-phase form (O_m = alpha_m rho e^{i phi_m} with D
 * independent phase maps, the paper's "TS" variables, Sec. 5); the auxiliary
 * variables of Eq. 8 (rho = mask e^{chi}, alpha_m = e^{alpha_t_m}, alpha_0 = 1)
 * with the chain rule to them; and the minibatch Adam iteration of Alg. 1
 * without its projector line (Adam as in Kingma and Ba, arXiv 1412.6980); and
 * that projector, Pi_U of Eq. 10, with a reliability-sorted 2-D phase
 * unwrapper written from Herraez et al. (2002).
 *
 * Complex arrays are interleaved (re, im) doubles.  Layouts (row-major):
 *   rho [n1][n2], u [C][n1][n2], alpha [D], G [D][C], scan [J][2] (row, col of
 *   the frame's top-left pixel), probe [Dp][M][M] (Dp = 1, D, or D*J when
 *   every frame has its own probe), y / bg / I [D][J][M][M]; frame index
 *   f = m*J + j.
 *
 * Scan positions off the pixel grid (Eq. 2's lateral shift S_j by a real
 * s_j = n_j + d_j, n_j integer, |d_j| <= 1/2): the exit wave sampled on the
 * object's pixels r = n_j + k is P(r - s_j) O(r) = P(k - d_j) O(n_j + k), so
 * frame j keeps the integer window n_j and takes the probe shifted by d_j,
 * P_d(k) = P(k - d) as the band-limited (Fourier) interpolation of P
 * (oracle_probe_shift); those probes enter as one probe per frame.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n1, n2;          /* object grid rows, columns                       */
    int ncomp;           /* displacement components C                       */
    int npeaks;          /* Bragg peaks D                                   */
    int m;               /* frame (and probe) side M                        */
    int nscan;           /* scan positions J per peak                       */
    const double *G;     /* [D][C] scattering vectors                       */
    const int *scan;     /* [J][2] top-left (row, col)                      */
    double phase_scale;  /* phi = phase_scale * G.u                         */
    int probe_per_peak;  /* 0: one probe for all peaks; 1: [D][M][M];       */
                         /* 2: one per frame, [D*J][M][M] (frame order)     */
} oracle_problem;

/* the probe of frame (peak mpk, scan j) */
static const double *frame_probe(const oracle_problem *p, const double *probe, int mpk, int j)
{
    long mm = (long)p->m * p->m;
    if (p->probe_per_peak == 2) return probe + ((long)mpk * p->nscan + j) * 2 * mm;
    return probe + (p->probe_per_peak ? (long)mpk * 2 * mm : 0);
}

typedef struct {
    double c_armijo;     /* sufficient-decrease constant                    */
    double grow;         /* step growth after an accepted step              */
    double shrink;       /* step shrink after a rejected step               */
    double t0;           /* initial step length                             */
    double w_rho, w_u, w_alpha; /* per-block step weights (diagonal scaling) */
} oracle_step_params;

typedef struct {
    double f_prev;       /* loss at the last accepted iterate               */
    double gn2_prev;     /* weighted squared gradient norm there            */
    double t;            /* step length of the current trial                */
    double f_last;       /* loss evaluated by the last call                 */
    int k;               /* number of calls so far                          */
    int accepted;        /* 1 if the last call accepted its iterate         */
    int n_accept, n_reject;
} oracle_step_state;

/* ------------------------------------------------------------------------ */
/* Direct DFT                                                               */
/* ------------------------------------------------------------------------ */

/* cos/sin(2 pi t / m) for t in [0, m): the DFT kernel takes its exponent
 * modulo M, so only these m values occur. */
static void twiddles(int m, double *ct, double *st)
{
    for (int t = 0; t < m; ++t) {
        double a = 2.0 * M_PI * (double)t / (double)m;
        ct[t] = cos(a);
        st[t] = sin(a);
    }
}

/* out(q0,q1) = sum_{k0,k1} in(k0,k1) exp(sign * 2 pi i (q0 k0 + q1 k1) / m).
 * sign = -1: the forward transform F of Eq. 2; sign = +1: F^H (no 1/m^2).
 * Separable: a direct sum along rows, then along columns. */
static void dft2_direct(int m, const double *in, double *out, int sign,
                        const double *ct, const double *st, double *tmp)
{
    for (int k0 = 0; k0 < m; ++k0) {
        for (int q1 = 0; q1 < m; ++q1) {
            double sr = 0.0, si = 0.0;
            for (int k1 = 0; k1 < m; ++k1) {
                int t = (q1 * k1) % m;
                double wr = ct[t], wi = sign * st[t];
                double xr = in[2 * (k0 * m + k1)], xi = in[2 * (k0 * m + k1) + 1];
                sr += xr * wr - xi * wi;
                si += xr * wi + xi * wr;
            }
            tmp[2 * (k0 * m + q1)] = sr;
            tmp[2 * (k0 * m + q1) + 1] = si;
        }
    }
    for (int q0 = 0; q0 < m; ++q0) {
        for (int q1 = 0; q1 < m; ++q1) {
            double sr = 0.0, si = 0.0;
            for (int k0 = 0; k0 < m; ++k0) {
                int t = (q0 * k0) % m;
                double wr = ct[t], wi = sign * st[t];
                double xr = tmp[2 * (k0 * m + q1)], xi = tmp[2 * (k0 * m + q1) + 1];
                sr += xr * wr - xi * wi;
                si += xr * wi + xi * wr;
            }
            out[2 * (q0 * m + q1)] = sr;
            out[2 * (q0 * m + q1) + 1] = si;
        }
    }
}

/* Exposed for the DFT pins: closed forms, Parseval, adjoint identity. */
void oracle_dft2(int m, const double *in, double *out, int sign)
{
    double *ct = malloc(sizeof(double) * m), *st = malloc(sizeof(double) * m);
    double *tmp = malloc(sizeof(double) * 2 * m * m);
    twiddles(m, ct, st);
    dft2_direct(m, in, out, sign, ct, st, tmp);
    free(ct); free(st); free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 / Eq. 3: the effective object of each Bragg peak                  */
/* ------------------------------------------------------------------------ */

static double phase_at(const oracle_problem *p, const double *u, int mpk, long r)
{
    long npix = (long)p->n1 * p->n2;
    double s = 0.0;
    for (int c = 0; c < p->ncomp; ++c)
        s += p->G[mpk * p->ncomp + c] * u[c * npix + r];
    return p->phase_scale * s;
}

void oracle_object_build(const oracle_problem *p, const double *rho, const double *u,
                         const double *alpha, double *O)
{
    long npix = (long)p->n1 * p->n2;
    for (int mpk = 0; mpk < p->npeaks; ++mpk) {
        for (long r = 0; r < npix; ++r) {
            double ph = phase_at(p, u, mpk, r);
            O[2 * (mpk * npix + r)] = alpha[mpk] * rho[r] * cos(ph);
            O[2 * (mpk * npix + r) + 1] = alpha[mpk] * rho[r] * sin(ph);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: exit wave of one frame and its far field                          */
/* ------------------------------------------------------------------------ */

/* psi(k) = P_m(k) * O_m(s_j + k), zero where s_j + k leaves the grid. */
static void exit_wave(const oracle_problem *p, const double *O, const double *probe,
                      int mpk, int j, double *psi)
{
    int m = p->m;
    long npix = (long)p->n1 * p->n2;
    const double *P = frame_probe(p, probe, mpk, j);
    int s0 = p->scan[2 * j], s1 = p->scan[2 * j + 1];
    for (int k0 = 0; k0 < m; ++k0) {
        for (int k1 = 0; k1 < m; ++k1) {
            int r0 = s0 + k0, r1 = s1 + k1;
            double zr = 0.0, zi = 0.0;
            if (r0 >= 0 && r0 < p->n1 && r1 >= 0 && r1 < p->n2) {
                long r = (long)r0 * p->n2 + r1;
                zr = O[2 * (mpk * npix + r)];
                zi = O[2 * (mpk * npix + r) + 1];
            }
            double pr = P[2 * (k0 * m + k1)], pi = P[2 * (k0 * m + k1) + 1];
            psi[2 * (k0 * m + k1)] = pr * zr - pi * zi;
            psi[2 * (k0 * m + k1) + 1] = pr * zi + pi * zr;
        }
    }
}

void oracle_forward(const oracle_problem *p, const double *rho, const double *u,
                    const double *alpha, const double *probe, const double *bg,
                    double *I)
{
    int m = p->m;
    long npix = (long)p->n1 * p->n2, mm = (long)m * m;
    double *O = malloc(sizeof(double) * 2 * p->npeaks * npix);
    oracle_object_build(p, rho, u, alpha, O);
    long nfr = (long)p->npeaks * p->nscan;
#pragma omp parallel
    {
        double *ct = malloc(sizeof(double) * m), *st = malloc(sizeof(double) * m);
        double *psi = malloc(sizeof(double) * 2 * mm), *Psi = malloc(sizeof(double) * 2 * mm);
        double *tmp = malloc(sizeof(double) * 2 * mm);
        twiddles(m, ct, st);
#pragma omp for schedule(static)
        for (long f = 0; f < nfr; ++f) {
            int mpk = (int)(f / p->nscan), j = (int)(f % p->nscan);
            exit_wave(p, O, probe, mpk, j, psi);
            dft2_direct(m, psi, Psi, -1, ct, st, tmp);
            for (long q = 0; q < mm; ++q) {
                double v = Psi[2 * q] * Psi[2 * q] + Psi[2 * q + 1] * Psi[2 * q + 1];
                I[f * mm + q] = v + (bg ? bg[f * mm + q] : 0.0);
            }
        }
        free(ct); free(st); free(psi); free(Psi); free(tmp);
    }
    free(O);
}

/* ------------------------------------------------------------------------ */
/* Eq. 4 and its gradient                                                   */
/* ------------------------------------------------------------------------ */

/* Loss and gradient over the frames listed in `frames` (all D*J frames when
 * frames == NULL), i.e. the minibatch sum of Eq. 11 with the minibatch given,
 * for objects O_m = alpha_m rho E_m with the phase factors E_m = e^{i phi_m}
 * given ([D][npix] complex).  Outputs (overwritten): g_rho, g_phi [D][npix]
 * (df/dphi_m), g_alpha.  frame_loss (nullable) receives each listed frame's
 * own term.  nthreads <= 0 uses the OpenMP default.  Returns the loss. */
static double loss_grad_core(const oracle_problem *p, const double *rho, const double *E,
                             const double *alpha, const double *probe, const double *bg,
                             const double *y, const int *frames, int nframes,
                             double *g_rho, double *g_phi_out, double *g_alpha,
                             double *frame_loss, int nthreads)
{
    int m = p->m, D = p->npeaks;
    long npix = (long)p->n1 * p->n2, mm = (long)m * m;
    long nlist = frames ? nframes : (long)D * p->nscan;
    double *O = malloc(sizeof(double) * 2 * D * npix);
    for (int mpk = 0; mpk < D; ++mpk)
        for (long r = 0; r < npix; ++r) {
            O[2 * (mpk * npix + r)] = alpha[mpk] * rho[r] * E[2 * (mpk * npix + r)];
            O[2 * (mpk * npix + r) + 1] = alpha[mpk] * rho[r] * E[2 * (mpk * npix + r) + 1];
        }

    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    /* per-thread accumulators, summed in thread order afterwards */
    double *t_loss = calloc(nt, sizeof(double));
    double *t_grho = calloc((size_t)nt * npix, sizeof(double));
    double *t_gphi = calloc((size_t)nt * D * npix, sizeof(double));
    double *t_galpha = calloc((size_t)nt * D, sizeof(double));

#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *ct = malloc(sizeof(double) * m), *st = malloc(sizeof(double) * m);
        double *psi = malloc(sizeof(double) * 2 * mm), *Psi = malloc(sizeof(double) * 2 * mm);
        double *chi = malloc(sizeof(double) * 2 * mm), *gh = malloc(sizeof(double) * 2 * mm);
        double *tmp = malloc(sizeof(double) * 2 * mm);
        double *grho = t_grho + (size_t)tid * npix;
        double *gphi = t_gphi + (size_t)tid * D * npix;
        double *galpha = t_galpha + (size_t)tid * D;
        twiddles(m, ct, st);
#pragma omp for schedule(static)
        for (long i = 0; i < nlist; ++i) {
            long f = frames ? frames[i] : i;
            int mpk = (int)(f / p->nscan), j = (int)(f % p->nscan);
            const double *P = frame_probe(p, probe, mpk, j);
            int s0 = p->scan[2 * j], s1 = p->scan[2 * j + 1];

            exit_wave(p, O, probe, mpk, j, psi);
            dft2_direct(m, psi, Psi, -1, ct, st, tmp);

            /* amplitude residual, loss term and chi = 2 df/dconj(Psi) */
            double fl = 0.0;
            for (long q = 0; q < mm; ++q) {
                double pr = Psi[2 * q], pi = Psi[2 * q + 1];
                double I = pr * pr + pi * pi + (bg ? bg[f * mm + q] : 0.0);
                double sI = sqrt(I);
                double res = sI - sqrt(y[f * mm + q]);
                fl += 0.5 * res * res;
                double sc = (I > 0.0) ? res / sI : 0.0;
                chi[2 * q] = sc * pr;
                chi[2 * q + 1] = sc * pi;
            }
            t_loss[tid] += fl;
            if (frame_loss) frame_loss[i] = fl;

            dft2_direct(m, chi, gh, +1, ct, st, tmp);   /* ghat = F^H chi */

            for (int k0 = 0; k0 < m; ++k0) {
                for (int k1 = 0; k1 < m; ++k1) {
                    int r0 = s0 + k0, r1 = s1 + k1;
                    if (r0 < 0 || r0 >= p->n1 || r1 < 0 || r1 >= p->n2) continue;
                    long r = (long)r0 * p->n2 + r1;
                    long kk = (long)k0 * m + k1;
                    /* g = conj(P) ghat ; cg = conj(g) = P conj(ghat) */
                    double Pr = P[2 * kk], Pi = P[2 * kk + 1];
                    double hr = gh[2 * kk], hi = gh[2 * kk + 1];
                    double gr = Pr * hr + Pi * hi;     /* Re(conj(P) ghat) */
                    double gi = Pr * hi - Pi * hr;     /* Im(conj(P) ghat) */
                    double cgr = gr, cgi = -gi;        /* conj(g) */
                    double er = E[2 * (mpk * npix + r)], ei = E[2 * (mpk * npix + r) + 1];
                    double orr = O[2 * (mpk * npix + r)], oi = O[2 * (mpk * npix + r) + 1];
                    double te_r = cgr * er - cgi * ei;         /* Re(conj(g) e) */
                    double to_i = cgr * oi + cgi * orr;        /* Im(conj(g) O) */
                    grho[r] += alpha[mpk] * te_r;
                    gphi[mpk * npix + r] += -to_i;
                    galpha[mpk] += rho[r] * te_r;
                }
            }
        }
        free(ct); free(st); free(psi); free(Psi); free(chi); free(gh); free(tmp);
    }

    double loss = 0.0;
    for (long r = 0; r < npix; ++r) g_rho[r] = 0.0;
    for (long r = 0; r < (long)D * npix; ++r) g_phi_out[r] = 0.0;
    for (int mpk = 0; mpk < D; ++mpk) g_alpha[mpk] = 0.0;
    for (int t = 0; t < nt; ++t) {
        loss += t_loss[t];
        for (long r = 0; r < npix; ++r) g_rho[r] += t_grho[(size_t)t * npix + r];
        for (long r = 0; r < (long)D * npix; ++r) g_phi_out[r] += t_gphi[(size_t)t * D * npix + r];
        for (int mpk = 0; mpk < D; ++mpk) g_alpha[mpk] += t_galpha[(size_t)t * D + mpk];
    }
    free(t_loss); free(t_grho); free(t_gphi); free(t_galpha);
    free(O);
    return loss;
}

/* e^{i phi} of per-peak phase maps phi [D][npix] */
static double *phase_factors(long n, const double *phi)
{
    double *E = malloc(sizeof(double) * 2 * n);
    for (long i = 0; i < n; ++i) {
        E[2 * i] = cos(phi[i]);
        E[2 * i + 1] = sin(phi[i]);
    }
    return E;
}

/* Eq. 4 and its gradient in the displacement form of Eq. 3: phi_m =
 * phase_scale * G_m . u, and df/du_c = phase_scale * sum_m G_{m,c} df/dphi_m.
 * Arguments as loss_grad_core, with u [C][n1][n2] and g_u [C][n1][n2]. */
double oracle_loss_grad(const oracle_problem *p, const double *rho, const double *u,
                        const double *alpha, const double *probe, const double *bg,
                        const double *y, const int *frames, int nframes,
                        double *g_rho, double *g_u, double *g_alpha,
                        double *frame_loss, int nthreads)
{
    int D = p->npeaks, C = p->ncomp;
    long npix = (long)p->n1 * p->n2;
    double *phi = malloc(sizeof(double) * D * npix);
    for (int mpk = 0; mpk < D; ++mpk)
        for (long r = 0; r < npix; ++r) phi[mpk * npix + r] = phase_at(p, u, mpk, r);
    double *E = phase_factors((long)D * npix, phi);
    double *gphi = malloc(sizeof(double) * D * npix);
    double loss = loss_grad_core(p, rho, E, alpha, probe, bg, y, frames, nframes, g_rho, gphi,
                                 g_alpha, frame_loss, nthreads);
    /* d phi_m / d u_c = phase_scale * G_{m,c} */
    for (int c = 0; c < C; ++c)
        for (long r = 0; r < npix; ++r) {
            double s = 0.0;
            for (int mpk = 0; mpk < D; ++mpk)
                s += p->G[mpk * C + c] * gphi[mpk * npix + r];
            g_u[c * npix + r] = p->phase_scale * s;
        }
    free(phi); free(E); free(gphi);
    return loss;
}

/* The per-peak-phase form (the paper's two-step "TS" reconstruction, Sec. 5):
 * O_m = alpha_m rho e^{i phi_m} with D independent phase maps phi [D][n1][n2]
 * in place of the displacement field; g_phi [D][n1][n2] = df/dphi_m. */
double oracle_loss_grad_phases(const oracle_problem *p, const double *rho, const double *phi,
                               const double *alpha, const double *probe, const double *bg,
                               const double *y, const int *frames, int nframes,
                               double *g_rho, double *g_phi, double *g_alpha, int nthreads)
{
    long n = (long)p->npeaks * p->n1 * p->n2;
    double *E = phase_factors(n, phi);
    double loss = loss_grad_core(p, rho, E, alpha, probe, bg, y, frames, nframes, g_rho, g_phi,
                                 g_alpha, NULL, nthreads);
    free(E);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1: the auxiliary variables of Eq. 8 and the Adam update             */
/* ------------------------------------------------------------------------ */

/* Eq. 4 and its gradient in the auxiliary variables of Eq. 8: rho = mask *
 * e^{chi} (mask [n1][n2] nullable = all ones: the support constraint),
 * alpha_0 = 1 (the reference peak) and alpha_m = e^{alpha_t[m]} for m >= 1.
 * g_chi = rho df/drho, g_alpha_t[m] = alpha_m df/dalpha_m (0 for m = 0),
 * g_u = df/du.  Returns the loss over the listed frames. */
double oracle_loss_grad_log(const oracle_problem *p, const double *chi, const double *u,
                            const double *alpha_t, const double *mask, const double *probe,
                            const double *bg, const double *y, const int *frames, int nframes,
                            double *g_chi, double *g_u, double *g_alpha_t, int nthreads)
{
    int D = p->npeaks;
    long npix = (long)p->n1 * p->n2;
    double *rho = malloc(sizeof(double) * npix);
    double *alpha = malloc(sizeof(double) * D);
    double *grho = malloc(sizeof(double) * npix);
    double *galpha = malloc(sizeof(double) * D);
    for (long r = 0; r < npix; ++r) rho[r] = (mask ? mask[r] : 1.0) * exp(chi[r]);
    alpha[0] = 1.0;
    for (int mpk = 1; mpk < D; ++mpk) alpha[mpk] = exp(alpha_t[mpk]);
    double loss = oracle_loss_grad(p, rho, u, alpha, probe, bg, y, frames, nframes, grho, g_u,
                                   galpha, NULL, nthreads);
    for (long r = 0; r < npix; ++r) g_chi[r] = rho[r] * grho[r];
    g_alpha_t[0] = 0.0;
    for (int mpk = 1; mpk < D; ++mpk) g_alpha_t[mpk] = alpha[mpk] * galpha[mpk];
    free(rho); free(alpha); free(grho); free(galpha);
    return loss;
}

/* Adam (Kingma and Ba, arXiv 1412.6980, Algorithm 1) on n variables x with
 * gradient g at step t >= 1 (the step count including this one):
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   x -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void oracle_adam_update(long n, double *x, const double *g, double *mo, double *ve, long t,
                        double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (long i = 0; i < n; ++i) {
        mo[i] = b1 * mo[i] + (1.0 - b1) * g[i];
        ve[i] = b2 * ve[i] + (1.0 - b2) * g[i] * g[i];
        x[i] -= lr * (mo[i] / c1) / (sqrt(ve[i] / c2) + eps);
    }
}

typedef struct {
    double lr_u, lr_chi, lr_alpha;   /* Adam step sizes of u, chi, alpha_t */
    double beta1, beta2, eps;
} oracle_adam_params;

/* One minibatch iteration of Alg. 1 without the projector (its line 5): the
 * gradient of Eq. 4 over the listed frames in the variables of Eq. 8, then
 * Adam on u, chi and alpha_t (alpha_t[0] is not a variable: its gradient is 0,
 * so it never moves).  *t counts the iterations (incremented here); the
 * moments [m, v] of each block are caller-owned and start at 0.  Returns the
 * minibatch loss at the iterate before the update. */
double oracle_adam_step(const oracle_problem *p, const double *probe, const double *bg,
                        const double *y, const int *frames, int nframes, const double *mask,
                        const oracle_adam_params *prm, long *t,
                        double *chi, double *u, double *alpha_t,
                        double *m_chi, double *v_chi, double *m_u, double *v_u,
                        double *m_a, double *v_a, int nthreads)
{
    int D = p->npeaks, C = p->ncomp;
    long npix = (long)p->n1 * p->n2;
    double *gchi = malloc(sizeof(double) * npix);
    double *gu = malloc(sizeof(double) * C * npix);
    double *ga = malloc(sizeof(double) * D);
    double f = oracle_loss_grad_log(p, chi, u, alpha_t, mask, probe, bg, y, frames, nframes,
                                    gchi, gu, ga, nthreads);
    *t += 1;
    oracle_adam_update(npix, chi, gchi, m_chi, v_chi, *t, prm->lr_chi, prm->beta1, prm->beta2, prm->eps);
    oracle_adam_update((long)C * npix, u, gu, m_u, v_u, *t, prm->lr_u, prm->beta1, prm->beta2, prm->eps);
    oracle_adam_update(D, alpha_t, ga, m_a, v_a, *t, prm->lr_alpha, prm->beta1, prm->beta2, prm->eps);
    free(gchi); free(gu); free(ga);
    return f;
}

/* ------------------------------------------------------------------------ */
/* One gradient-descent iteration with a lagged Armijo line search          */
/* ------------------------------------------------------------------------ */

/* The optimizer iteration around the loss and gradient (the place of the
 * update in Alg. 1; plain gradient descent instead of Adam):
 *   1. f, g at the current iterate x.
 *   2. Accept x when it is the first call, or when f is finite and
 *      f <= f_prev - c * t * gn2_prev  (sufficient decrease along -w*g_prev).
 *   3. Accepted: x_prev = x, g_prev = g, f_prev = f, gn2_prev = sum_b w_b |g_b|^2,
 *      and t = grow * t (not on the first call).  Rejected: t = shrink * t.
 *   4. x = x_prev - t * w * g_prev.  alpha_0 (the reference peak's scaling) is
 *      not a variable: it is neither updated nor counted in gn2.
 * x_prev and g_prev are caller-owned buffers of the same shapes as rho, u, alpha. */
void oracle_step(const oracle_problem *p, const double *probe, const double *bg,
                 const double *y, const oracle_step_params *prm, oracle_step_state *st,
                 double *rho, double *u, double *alpha,
                 double *rho_prev, double *u_prev, double *alpha_prev,
                 double *grho_prev, double *gu_prev, double *galpha_prev, int nthreads)
{
    int D = p->npeaks, C = p->ncomp;
    long npix = (long)p->n1 * p->n2;
    double *grho = malloc(sizeof(double) * npix);
    double *gu = malloc(sizeof(double) * C * npix);
    double *galpha = malloc(sizeof(double) * D);
    double f = oracle_loss_grad(p, rho, u, alpha, probe, bg, y, NULL, 0,
                                grho, gu, galpha, NULL, nthreads);
    int accept;
    if (st->k == 0)
        accept = isfinite(f);
    else
        accept = isfinite(f) && (f <= st->f_prev - prm->c_armijo * st->t * st->gn2_prev);
    if (accept) {
        double gn2 = 0.0, a = 0.0, b = 0.0, c = 0.0;
        for (long r = 0; r < npix; ++r) a += grho[r] * grho[r];
        for (long r = 0; r < (long)C * npix; ++r) b += gu[r] * gu[r];
        for (int mpk = 1; mpk < D; ++mpk) c += galpha[mpk] * galpha[mpk];
        gn2 = prm->w_rho * a + prm->w_u * b + prm->w_alpha * c;
        memcpy(rho_prev, rho, sizeof(double) * npix);
        memcpy(u_prev, u, sizeof(double) * C * npix);
        memcpy(alpha_prev, alpha, sizeof(double) * D);
        memcpy(grho_prev, grho, sizeof(double) * npix);
        memcpy(gu_prev, gu, sizeof(double) * C * npix);
        memcpy(galpha_prev, galpha, sizeof(double) * D);
        if (st->k > 0) st->t *= prm->grow;
        st->f_prev = f;
        st->gn2_prev = gn2;
        st->n_accept += 1;
    } else {
        st->t *= prm->shrink;
        st->n_reject += 1;
    }
    st->accepted = accept;
    st->f_last = f;
    for (long r = 0; r < npix; ++r)
        rho[r] = rho_prev[r] - st->t * prm->w_rho * grho_prev[r];
    for (long r = 0; r < (long)C * npix; ++r)
        u[r] = u_prev[r] - st->t * prm->w_u * gu_prev[r];
    alpha[0] = alpha_prev[0];
    for (int mpk = 1; mpk < D; ++mpk)
        alpha[mpk] = alpha_prev[mpk] - st->t * prm->w_alpha * galpha_prev[mpk];
    st->k += 1;
    free(grho); free(gu); free(galpha);
}

/* ------------------------------------------------------------------------ */
/* Eq. 9 / Eq. 10: phase wrapping, 2-D unwrapping, the projector Pi_U       */
/* ------------------------------------------------------------------------ */

static const double TWO_PI = 6.283185307179586476925286766559;

/* W: the wrapped value of x in [-pi, pi) */
static double wrap_phase(double x)
{
    return x - TWO_PI * floor(x / TWO_PI + 0.5);
}

typedef struct { double w; long id; } unwrap_edge;

/* descending reliability, then ascending edge number: a strict total order */
static int edge_cmp(const void *a, const void *b)
{
    const unwrap_edge *x = a, *y = b;
    if (x->w > y->w) return -1;
    if (x->w < y->w) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* 2-D phase unwrapping by reliability-sorted, non-continuous path following
 * (Herraez, Burton, Lalor and Gdeisat, Appl. Opt. 41, 7437 (2002)), written
 * from that description in the plainest form:
 *   reliability R = 1 / D of a pixel whose eight neighbours are inside the
 *     grid and the mask, D^2 = H^2 + V^2 + D1^2 + D2^2 with the second
 *     differences H, V, D1, D2 of the wrapped phase along the two axes and
 *     the two diagonals (each first difference wrapped); R = 0 elsewhere;
 *   an edge joins two 4-neighbours in the mask, with reliability R_p + R_q;
 *   edges are taken in order of decreasing reliability (ties: lower edge
 *     number first; edge 2r joins pixel r to its right neighbour, 2r + 1 to
 *     the one below); when an edge joins two groups, the group of its second
 *     pixel is shifted by the multiple of 2 pi that brings the difference
 *     across the edge into [-pi, pi), and the groups merge.
 * Finally every group is shifted by the multiple of 2 pi that gives its
 * lowest-numbered pixel back its wrapped value (so the result is unique for
 * data without residues).  Pixels off the mask keep their wrapped value.
 * mask (nullable = all pixels) is [n1][n2] with nonzero = inside. */
void oracle_unwrap2d(int n1, int n2, const double *wrapped, const double *mask, double *out)
{
    long n = (long)n1 * n2;
    double *R = calloc(n, sizeof(double));
    long *label = malloc(sizeof(long) * n);
    unwrap_edge *e = malloc(sizeof(unwrap_edge) * 2 * n);
#define IN(i, j) ((i) >= 0 && (i) < n1 && (j) >= 0 && (j) < n2 && (!mask || mask[(long)(i) * n2 + (j)] != 0.0))
#define PH(i, j) wrapped[(long)(i) * n2 + (j)]
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j) {
            int ok = 1;
            for (int di = -1; di <= 1; ++di)
                for (int dj = -1; dj <= 1; ++dj)
                    ok = ok && IN(i + di, j + dj);
            if (!ok) continue;
            double c = PH(i, j);
            double h = wrap_phase(PH(i, j - 1) - c) - wrap_phase(c - PH(i, j + 1));
            double v = wrap_phase(PH(i - 1, j) - c) - wrap_phase(c - PH(i + 1, j));
            double d1 = wrap_phase(PH(i - 1, j - 1) - c) - wrap_phase(c - PH(i + 1, j + 1));
            double d2 = wrap_phase(PH(i - 1, j + 1) - c) - wrap_phase(c - PH(i + 1, j - 1));
            double dd = sqrt(h * h + v * v + d1 * d1 + d2 * d2);
            R[(long)i * n2 + j] = 1.0 / (dd > 1e-300 ? dd : 1e-300);
        }
    long ne = 0;
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j) {
            long r = (long)i * n2 + j;
            if (!IN(i, j)) continue;
            if (IN(i, j + 1)) { e[ne].w = R[r] + R[r + 1]; e[ne].id = 2 * r; ++ne; }
            if (IN(i + 1, j)) { e[ne].w = R[r] + R[r + n2]; e[ne].id = 2 * r + 1; ++ne; }
        }
    qsort(e, ne, sizeof(unwrap_edge), edge_cmp);
    for (long r = 0; r < n; ++r) { out[r] = wrapped[r]; label[r] = r; }
    for (long k = 0; k < ne; ++k) {
        long pa = e[k].id / 2;
        long pb = (e[k].id & 1) ? pa + n2 : pa + 1;
        long la = label[pa], lb = label[pb];
        if (la == lb) continue;
        double shift = TWO_PI * floor((out[pa] - out[pb]) / TWO_PI + 0.5);
        for (long r = 0; r < n; ++r)
            if (label[r] == lb) { out[r] += shift; label[r] = la; }
    }
    /* each group's lowest-numbered pixel keeps its wrapped value */
    for (long r = 0; r < n; ++r) {
        if (label[r] < 0) continue;                 /* group already normalised */
        long l = label[r];
        double shift = wrapped[r] - out[r];
        for (long q = r; q < n; ++q)
            if (label[q] == l) { out[q] += shift; label[q] = -1; }
    }
#undef IN
#undef PH
    free(R); free(label); free(e);
}

/* Moore-Penrose pseudo-inverse pinv [C][D] of G [D][C] (C <= 3) through the
 * eigen-decomposition of G^T G by cyclic Jacobi rotations; eigenvalues below
 * 1e-12 of the largest count as zero. */
static void pinv_g(int D, int C, const double *G, double *pinv)
{
    double A[3][3] = {{0}}, V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int a = 0; a < C; ++a)
        for (int b = 0; b < C; ++b)
            for (int m = 0; m < D; ++m) A[a][b] += G[m * C + a] * G[m * C + b];
    for (int sweep = 0; sweep < 50; ++sweep)
        for (int pq = 0; pq < C; ++pq)
            for (int qq = pq + 1; qq < C; ++qq) {
                if (fabs(A[pq][qq]) < 1e-300) continue;
                double th = 0.5 * atan2(2 * A[pq][qq], A[qq][qq] - A[pq][pq]);
                double c = cos(th), sn = sin(th);
                for (int k = 0; k < C; ++k) {         /* A = J^T A J */
                    double akp = A[k][pq], akq = A[k][qq];
                    A[k][pq] = c * akp - sn * akq;
                    A[k][qq] = sn * akp + c * akq;
                }
                for (int k = 0; k < C; ++k) {
                    double apk = A[pq][k], aqk = A[qq][k];
                    A[pq][k] = c * apk - sn * aqk;
                    A[qq][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < C; ++k) {
                    double vkp = V[k][pq], vkq = V[k][qq];
                    V[k][pq] = c * vkp - sn * vkq;
                    V[k][qq] = sn * vkp + c * vkq;
                }
            }
    double lmax = 0.0;
    for (int a = 0; a < C; ++a) lmax = fmax(lmax, fabs(A[a][a]));
    double Ainv[3][3] = {{0}};
    for (int a = 0; a < C; ++a)
        for (int b = 0; b < C; ++b)
            for (int k = 0; k < C; ++k)
                if (A[k][k] > 1e-12 * lmax) Ainv[a][b] += V[a][k] * V[b][k] / A[k][k];
    for (int a = 0; a < C; ++a)
        for (int m = 0; m < D; ++m) {
            double s = 0.0;
            for (int b = 0; b < C; ++b) s += Ainv[a][b] * G[m * C + b];
            pinv[a * D + m] = s;
        }
}

/* Pi_U of Eq. 10: phases Phi_m = phase_scale G_m . u, wrapped (Eq. 9's W),
 * unwrapped per peak inside the mask, and mapped back to u by the
 * pseudo-inverse of G (the (H H^T)^{-1} H of Eq. 9 when the G_m span the
 * components of u).  Written as a correction, u_out = u + (Phi' - Phi) G^+^T /
 * phase_scale, so that components outside the span of the G_m (u_z for
 * in-plane peaks) are left as they are.  Pixels off the mask are unchanged. */
void oracle_project_u(const oracle_problem *p, const double *u, const double *mask, double *u_out)
{
    int D = p->npeaks, C = p->ncomp;
    long npix = (long)p->n1 * p->n2;
    double *phi = malloc(sizeof(double) * npix), *wr = malloc(sizeof(double) * npix);
    double *un = malloc(sizeof(double) * npix), *dphi = malloc(sizeof(double) * D * npix);
    double pinv[3 * 16];
    pinv_g(D, C, p->G, pinv);
    for (int m = 0; m < D; ++m) {
        for (long r = 0; r < npix; ++r) {
            phi[r] = phase_at(p, u, m, r);
            wr[r] = wrap_phase(phi[r]);
        }
        oracle_unwrap2d(p->n1, p->n2, wr, mask, un);
        for (long r = 0; r < npix; ++r) dphi[m * npix + r] = un[r] - phi[r];
    }
    for (int c = 0; c < C; ++c)
        for (long r = 0; r < npix; ++r) {
            double s = 0.0;
            if (!mask || mask[r] != 0.0)
                for (int m = 0; m < D; ++m) s += pinv[c * D + m] * dphi[m * npix + r];
            u_out[c * npix + r] = u[c * npix + r] + s / p->phase_scale;
        }
    free(phi); free(wr); free(un); free(dphi);
}

/* The illumination of Eq. 8's closing remark: out(r) = sum over every frame
 * (peak m, scan j) of |P_m(r - s_j)|^2 where r - s_j lies in the frame,
 * on the object grid [n1][n2] (overwritten).  The reconstruction's final
 * threshold sets the density to zero where this is small. */
void oracle_illumination(const oracle_problem *p, const double *probe, double *out)
{
    int m = p->m;
    long npix = (long)p->n1 * p->n2, mm = (long)m * m;
    for (long r = 0; r < npix; ++r) out[r] = 0.0;
    for (int mpk = 0; mpk < p->npeaks; ++mpk) {
        for (int j = 0; j < p->nscan; ++j) {
            const double *P = frame_probe(p, probe, mpk, j);
            for (int k0 = 0; k0 < m; ++k0)
                for (int k1 = 0; k1 < m; ++k1) {
                    int r0 = p->scan[2 * j] + k0, r1 = p->scan[2 * j + 1] + k1;
                    if (r0 < 0 || r0 >= p->n1 || r1 < 0 || r1 >= p->n2) continue;
                    long kk = (long)k0 * m + k1;
                    out[(long)r0 * p->n2 + r1] += P[2 * kk] * P[2 * kk] + P[2 * kk + 1] * P[2 * kk + 1];
                }
        }
    }
}

/* P_d(k) = P(k - d) for a probe [M][M] and a real offset d = (d0, d1): the
 * band-limited interpolation, by its definition through the DFT,
 *   P_d(k) = (1/M^2) sum_q Phat(q) exp(2 pi i q.(k - d)/M),  Phat = F P,
 * with each frequency component q taken in [-M/2, M/2).  out [M][M]
 * (interleaved complex, overwritten). */
void oracle_probe_shift(int m, const double *P, double d0, double d1, double *out)
{
    long mm = (long)m * m;
    double *ct = malloc(sizeof(double) * m), *st = malloc(sizeof(double) * m);
    double *Ph = malloc(sizeof(double) * 2 * mm), *tmp = malloc(sizeof(double) * 2 * mm);
    twiddles(m, ct, st);
    dft2_direct(m, P, Ph, -1, ct, st, tmp);
    for (int q0 = 0; q0 < m; ++q0)
        for (int q1 = 0; q1 < m; ++q1) {
            double f0 = q0 < m / 2 ? q0 : q0 - m, f1 = q1 < m / 2 ? q1 : q1 - m;
            double a = -2.0 * M_PI * (f0 * d0 + f1 * d1) / (double)m;
            double c = cos(a), sn = sin(a);
            long q = (long)q0 * m + q1;
            double xr = Ph[2 * q], xi = Ph[2 * q + 1];
            Ph[2 * q] = xr * c - xi * sn;
            Ph[2 * q + 1] = xr * sn + xi * c;
        }
    dft2_direct(m, Ph, out, +1, ct, st, tmp);
    for (long i = 0; i < 2 * mm; ++i) out[i] /= (double)mm;
    free(ct); free(st); free(Ph); free(tmp);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
