/*
 * oracle.c - plain, slow CPU FP64 oracle for bus injections and the
 * power-flow Jacobian, written from "Bus Admittance Matrix Revisited: Is It
 * Outdated on Modern Computers?" (Cui, arXiv 2302.10736).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path calls this file:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header or table with the CUDA library and must be
 * compiled with -ffp-contract=off so every product and sum rounds as written.
 *
 * Conventions (the paper's, Sec. II):
 *   branch l joins h = from[l] and k = to[l]; series admittance
 *   y_hk = g + j b; total line charging b_sh split as y_h = y_k = j b_sh / 2;
 *   off-nominal tap m e^{j phi} on the primary (h) side (Eqs. 5-6).
 *   Bus shunt y_sh,i = g_s,i + j b_s,i: Eq. 7 has no shunt term, and this
 *   file adds the shunt as a one-terminal element v_i^2 conj(y_sh,i) (its
 *   Ybus stamp is Y_ii += y_sh,i).
 *   V_i = v_i e^{j theta_i}; S = P + j Q.
 *   J = [[Re dS/dtheta, Re dS/dv], [Im dS/dtheta, Im dS/dv]] (Eq. 2) with the
 *   canonical CSR layout: P-row i holds the Ybus row-i columns j (theta
 *   columns) followed by nb + j (magnitude columns); Q-row nb+i repeats the
 *   structure 2*nnzY entries later.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (closed forms, circuit-law currents, complex-step derivatives, invariants,
 * brute-force dense evaluation, central differences).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------- Ybus ------ */

typedef struct {
    int row, col;
    long order; /* insertion order: fixes the summation order of duplicates */
    double re, im;
} or_trip;

static int or_trip_cmp(const void *a, const void *b)
{
    const or_trip *p = (const or_trip *)a, *q = (const or_trip *)b;
    if (p->row != q->row) return p->row < q->row ? -1 : 1;
    if (p->col != q->col) return p->col < q->col ? -1 : 1;
    return p->order < q->order ? -1 : (p->order > q->order);
}

/*
 * Bus admittance matrix in CSR (sorted columns, duplicates merged, every
 * diagonal present even when it is zero; explicit zeros kept, Sec. IV-B.2).
 * The four stamps of branch l are the pi-model whose terminal powers are
 * Eqs. (5)-(6):  Y_hh += (y_hk + y_h)/m^2,  Y_hk += -y_hk e^{j phi}/m,
 *                Y_kh += -y_hk e^{-j phi}/m,  Y_kk += y_hk + y_k.
 * Branches with skip[l] != 0 are left out (an N-1 contingency grid).
 * gs/bs may be NULL.  Arrays rp [nb+1], ci/yre/yim [nb + 2*nl].
 * Returns nnz, or -1 on allocation failure.
 */
int or_ybus(int nb, int nl, const int *from, const int *to, const double *g, const double *b,
            const double *bsh, const double *tap, const double *shift, const double *gs,
            const double *bs, const unsigned char *skip, int *rp, int *ci, double *yre, double *yim)
{
    long cap = (long)nb + 4L * nl;
    or_trip *tr = (or_trip *)malloc(sizeof(or_trip) * (size_t)(cap > 0 ? cap : 1));
    if (!tr) return -1;
    long n = 0;
    for (int i = 0; i < nb; ++i) {
        tr[n].row = i;
        tr[n].col = i;
        tr[n].order = n;
        tr[n].re = gs ? gs[i] : 0.0;
        tr[n].im = bs ? bs[i] : 0.0;
        ++n;
    }
    for (int l = 0; l < nl; ++l) {
        if (skip && skip[l]) continue;
        int h = from[l], k = to[l];
        cplx ys = g[l] + I * b[l];
        cplx ysh = I * (bsh[l] / 2.0);
        double m = tap[l];
        cplx eph = cexp(I * shift[l]);
        cplx yhh = (ys + ysh) / (m * m);
        cplx yhk = -ys * eph / m;
        cplx ykh = -ys * conj(eph) / m;
        cplx ykk = ys + ysh;
        int rr[4] = {h, h, k, k}, cc[4] = {h, k, h, k};
        cplx vv[4] = {yhh, yhk, ykh, ykk};
        for (int q = 0; q < 4; ++q) {
            tr[n].row = rr[q];
            tr[n].col = cc[q];
            tr[n].order = n;
            tr[n].re = creal(vv[q]);
            tr[n].im = cimag(vv[q]);
            ++n;
        }
    }
    qsort(tr, (size_t)n, sizeof(or_trip), or_trip_cmp);
    int nnz = 0;
    for (int i = 0; i <= nb; ++i) rp[i] = 0;
    for (long e = 0; e < n; ++e) {
        if (nnz > 0 && ci[nnz - 1] == tr[e].col && e > 0 && tr[e - 1].row == tr[e].row) {
            yre[nnz - 1] += tr[e].re;
            yim[nnz - 1] += tr[e].im;
        } else {
            ci[nnz] = tr[e].col;
            yre[nnz] = tr[e].re;
            yim[nnz] = tr[e].im;
            rp[tr[e].row + 1]++;
            ++nnz;
        }
    }
    for (int i = 0; i < nb; ++i) rp[i + 1] += rp[i];
    free(tr);
    return nnz;
}

/* Dense Ybus [nb*nb] (row-major) from the same stamps, for the tiny-grid tier. */
void or_ybus_dense(int nb, int nl, const int *from, const int *to, const double *g, const double *b,
                   const double *bsh, const double *tap, const double *shift, const double *gs,
                   const double *bs, double *Yre, double *Yim)
{
    for (long e = 0; e < (long)nb * nb; ++e) {
        Yre[e] = 0.0;
        Yim[e] = 0.0;
    }
    for (int i = 0; i < nb; ++i) {
        Yre[(long)i * nb + i] += gs ? gs[i] : 0.0;
        Yim[(long)i * nb + i] += bs ? bs[i] : 0.0;
    }
    for (int l = 0; l < nl; ++l) {
        int h = from[l], k = to[l];
        cplx ys = g[l] + I * b[l];
        cplx ysh = I * (bsh[l] / 2.0);
        double m = tap[l];
        cplx eph = cexp(I * shift[l]);
        cplx v[4] = {(ys + ysh) / (m * m), -ys * eph / m, -ys * conj(eph) / m, ys + ysh};
        long pos[4] = {(long)h * nb + h, (long)h * nb + k, (long)k * nb + h, (long)k * nb + k};
        for (int q = 0; q < 4; ++q) {
            Yre[pos[q]] += creal(v[q]);
            Yim[pos[q]] += cimag(v[q]);
        }
    }
}

/* ------------------------------------------------------ injections ------- */

/* Eq. (1) with a dense Ybus: S = V . conj(Y V). */
void or_inj_dense(int nb, const double *Yre, const double *Yim, const double *vm, const double *va,
                  double *P, double *Q)
{
    for (int i = 0; i < nb; ++i) {
        cplx Ii = 0.0;
        for (int j = 0; j < nb; ++j) {
            cplx Vj = vm[j] * cexp(I * va[j]);
            Ii += (Yre[(long)i * nb + j] + I * Yim[(long)i * nb + j]) * Vj;
        }
        cplx S = vm[i] * cexp(I * va[i]) * conj(Ii);
        P[i] = creal(S);
        Q[i] = cimag(S);
    }
}

/* Eq. (1) on the CSR Ybus, following Sec. IV-B.1: (1) U = e^{j theta},
   V = v U; (2) I = Ybus V; (3) S = V . conj(I). */
void or_inj_sparse(int nb, const int *rp, const int *ci, const double *yre, const double *yim,
                   const double *vm, const double *va, double *P, double *Q)
{
    cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)(nb > 0 ? nb : 1));
    for (int i = 0; i < nb; ++i) V[i] = vm[i] * cexp(I * va[i]);
    for (int i = 0; i < nb; ++i) {
        cplx Ii = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) Ii += (yre[e] + I * yim[e]) * V[ci[e]];
        cplx S = V[i] * conj(Ii);
        P[i] = creal(S);
        Q[i] = cimag(S);
    }
    free(V);
}

/* ------------------------------------------------------- Jacobian -------- */

/* Canonical J pattern (Eq. 2 block order) from the Ybus pattern.
   jrp [2nb+1], jci [4 nnzY]. */
void or_jac_pattern(int nb, const int *rp, const int *ci, int *jrp, int *jci)
{
    int nnz = rp[nb];
    for (int blk = 0; blk < 2; ++blk) {
        for (int i = 0; i < nb; ++i) {
            int d = rp[i + 1] - rp[i];
            int base = 2 * nnz * blk + 2 * rp[i];
            jrp[blk * nb + i] = base;
            for (int k = 0; k < d; ++k) {
                jci[base + k] = ci[rp[i] + k];
                jci[base + d + k] = nb + ci[rp[i] + k];
            }
        }
    }
    jrp[2 * nb] = 4 * nnz;
}

/* position of structural entry (i, j) within Ybus row i, or -1 */
static int or_find(const int *rp, const int *ci, int i, int j)
{
    for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] == j) return e - rp[i];
    return -1;
}

/* store the complex derivative pair at (i, j): d/dtheta_j and d/dv_j */
static void or_put(double *J, int nb, const int *rp, int i, int kpos, cplx dth, cplx dv)
{
    int nnz = rp[nb];
    int d = rp[i + 1] - rp[i];
    int p = 2 * rp[i] + kpos;
    J[p] = creal(dth);           /* J11 */
    J[p + d] = creal(dv);        /* J12 */
    J[2 * nnz + p] = cimag(dth);     /* J21 */
    J[2 * nnz + p + d] = cimag(dv);  /* J22 */
}

/*
 * Analytic Jacobian of the Ybus method on its own pattern, Eqs. (3)-(4):
 *   dS/dtheta = j diag(V) [diag(conj I) - conj(Ybus diag V)]
 *   dS/dv     = diag(conj(I) e^{j theta}) + diag(V) conj(Ybus diag e^{j theta})
 * entry by entry: for structural (i, j)
 *   dS_i/dtheta_j = -j V_i conj(Y_ij V_j) + [i == j] j V_i conj(I_i)
 *   dS_i/dv_j     =  V_i conj(Y_ij U_j)   + [i == j] conj(I_i) U_i
 * (Alg. 1 as printed differs from Eq. 3 by a sign; Eq. 3 is followed.)
 */
void or_jac_ybus(int nb, const int *rp, const int *ci, const double *yre, const double *yim,
                 const double *vm, const double *va, double *J)
{
    cplx *U = (cplx *)malloc(sizeof(cplx) * (size_t)(nb > 0 ? nb : 1));
    cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)(nb > 0 ? nb : 1));
    cplx *Ib = (cplx *)malloc(sizeof(cplx) * (size_t)(nb > 0 ? nb : 1));
    for (int i = 0; i < nb; ++i) {
        U[i] = cexp(I * va[i]);
        V[i] = vm[i] * U[i];
    }
    for (int i = 0; i < nb; ++i) {
        Ib[i] = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) Ib[i] += (yre[e] + I * yim[e]) * V[ci[e]];
    }
    for (int i = 0; i < nb; ++i) {
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int j = ci[e];
            cplx Y = yre[e] + I * yim[e];
            cplx dth = -I * V[i] * conj(Y * V[j]);
            cplx dv = V[i] * conj(Y * U[j]);
            if (i == j) {
                dth += I * V[i] * conj(Ib[i]);
                dv += conj(Ib[i]) * U[i];
            }
            or_put(J, nb, rp, i, e - rp[i], dth, dv);
        }
    }
    free(U);
    free(V);
    free(Ib);
}

/* real-form injection of row i (P + jQ with P = v_i sum v_k (G c + B s),
   Q = v_i sum v_k (G s - B c), c/s of theta_i - theta_k), evaluated in complex
   arithmetic so one coordinate can carry an imaginary step. */
static void or_row_realform(const int *rp, const int *ci, const double *yre, const double *yim, int i,
                            const cplx *vc, const cplx *tc, cplx *Pi, cplx *Qi)
{
    cplx p = 0.0, q = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int k = ci[e];
        cplx d = tc[i] - tc[k];
        cplx c = ccos(d), s = csin(d);
        p += vc[k] * (yre[e] * c + yim[e] * s);
        q += vc[k] * (yre[e] * s - yim[e] * c);
    }
    *Pi = vc[i] * p;
    *Qi = vc[i] * q;
}

/*
 * Jacobian by complex-step differentiation of the real-form injections
 * (Squire & Trapp 1998): dF/dx = Im F(x + i h) / h with h = 1e-30.  No
 * subtraction is involved, so the result is exact to rounding and pins every
 * structural entry of Eqs. (3)-(4) independently of their closed forms.
 */
void or_jac_cstep(int nb, const int *rp, const int *ci, const double *yre, const double *yim,
                  const double *vm, const double *va, double *J)
{
    const double h = 1e-30;
    cplx *vc = (cplx *)malloc(sizeof(cplx) * (size_t)(nb > 0 ? nb : 1));
    cplx *tc = (cplx *)malloc(sizeof(cplx) * (size_t)(nb > 0 ? nb : 1));
    for (int i = 0; i < nb; ++i) {
        vc[i] = vm[i];
        tc[i] = va[i];
    }
    for (int j = 0; j < nb; ++j) {
        /* rows with a structural entry in column j: the pattern is symmetric */
        for (int e = rp[j]; e < rp[j + 1]; ++e) {
            int i = ci[e];
            int kpos = or_find(rp, ci, i, j);
            cplx P1, Q1, P2, Q2;
            tc[j] = va[j] + I * h;
            or_row_realform(rp, ci, yre, yim, i, vc, tc, &P1, &Q1);
            tc[j] = va[j];
            vc[j] = vm[j] + I * h;
            or_row_realform(rp, ci, yre, yim, i, vc, tc, &P2, &Q2);
            vc[j] = vm[j];
            or_put(J, nb, rp, i, kpos, cimag(P1) / h + I * (cimag(Q1) / h), cimag(P2) / h + I * (cimag(Q2) / h));
        }
    }
    free(vc);
    free(tc);
}

/* ------------------------------------------------- element-wise method --- */

/*
 * Element-wise method, Sec. II-B and Sec. IV-C, in the paper's two steps.
 *
 * Evaluation (per line, Eqs. 5-6 and the 16 partials of P_h, Q_h, P_k, Q_k
 * with respect to v_h, theta_h, v_k, theta_k):
 *   S_hk = v_h^2 conj(y_h + y_hk)/m^2 - v_h v_k conj(y_hk)/m e^{j(th_h - th_k - phi)}
 *   S_kh = -v_h v_k conj(y_hk)/m e^{-j(th_h - th_k - phi)} + v_k^2 conj(y_k + y_hk)
 * Writing the coupling terms X_h = -v_h v_k conj(y_hk)/m e^{j(d - phi)} and
 * X_k = -v_h v_k conj(y_hk)/m e^{-j(d - phi)}, d = th_h - th_k:
 *   dS_hk/dth_h =  j X_h     dS_hk/dth_k = -j X_h
 *   dS_hk/dv_h  = 2 v_h conj(y_h + y_hk)/m^2 + X_h / v_h
 *   dS_hk/dv_k  = X_h / v_k
 *   dS_kh/dth_h = -j X_k     dS_kh/dth_k =  j X_k
 *   dS_kh/dv_h  = X_k / v_h
 *   dS_kh/dv_k  = 2 v_k conj(y_k + y_hk) + X_k / v_k
 * (derived from Eqs. 5-6; the paper states only that there are 16 of them.)
 *
 * Reduction (Eq. 7 and the copy-add of Fig. 2): bus powers are the sums of
 * the terminal powers of all incident lines (parallel lines separately) plus
 * the bus-shunt terminal v_i^2 conj(y_sh,i); each partial is added into the
 * Jacobian slot of its (row bus, column bus) pair on the Ybus pattern given
 * by rp/ci (which must be the pattern of the same branch set).
 * Branches with skip[l] != 0 are left out.  J may be NULL (powers only).
 * Returns the number of element partial values evaluated (16 per line).
 */
long or_elementwise(int nb, int nl, const int *from, const int *to, const double *g, const double *b,
                    const double *bsh, const double *tap, const double *shift, const double *gs,
                    const double *bs, const unsigned char *skip, const double *vm, const double *va,
                    const int *rp, const int *ci, double *P, double *Q, double *J)
{
    /* evaluation step: element arrays (S per terminal, 16 partials per line) */
    cplx *Sh = (cplx *)malloc(sizeof(cplx) * (size_t)(nl > 0 ? nl : 1));
    cplx *Sk = (cplx *)malloc(sizeof(cplx) * (size_t)(nl > 0 ? nl : 1));
    cplx *dS = (cplx *)malloc(sizeof(cplx) * (size_t)(nl > 0 ? 8 * nl : 1));
    long nvalues = 0;
    for (int l = 0; l < nl; ++l) {
        if (skip && skip[l]) continue;
        nvalues += 16; /* 8 complex partials = 16 real values (P and Q parts) */
        int h = from[l], k = to[l];
        double vh = vm[h], vk = vm[k], m = tap[l];
        cplx yhk = g[l] + I * b[l];
        cplx yh = I * (bsh[l] / 2.0), yk = yh;
        double d = va[h] - va[k];
        cplx Xh = -vh * vk * conj(yhk) / m * cexp(I * (d - shift[l]));
        cplx Xk = -vh * vk * conj(yhk) / m * cexp(-I * (d - shift[l]));
        Sh[l] = vh * vh * conj(yh + yhk) / (m * m) + Xh;
        Sk[l] = Xk + vk * vk * conj(yk + yhk);
        cplx *p = dS + 8 * (long)l;
        p[0] = I * Xh;                                      /* dS_hk/dth_h */
        p[1] = 2.0 * vh * conj(yh + yhk) / (m * m) + Xh / vh; /* dS_hk/dv_h */
        p[2] = -I * Xh;                                     /* dS_hk/dth_k */
        p[3] = Xh / vk;                                     /* dS_hk/dv_k */
        p[4] = -I * Xk;                                     /* dS_kh/dth_h */
        p[5] = Xk / vh;                                     /* dS_kh/dv_h */
        p[6] = I * Xk;                                      /* dS_kh/dth_k */
        p[7] = 2.0 * vk * conj(yk + yhk) + Xk / vk;         /* dS_kh/dv_k */
    }

    /* reduction step: powers onto buses */
    for (int i = 0; i < nb; ++i) {
        cplx ysh = (gs ? gs[i] : 0.0) + I * (bs ? bs[i] : 0.0);
        cplx S = vm[i] * vm[i] * conj(ysh);
        P[i] = creal(S);
        Q[i] = cimag(S);
    }
    for (int l = 0; l < nl; ++l) {
        if (skip && skip[l]) continue;
        P[from[l]] += creal(Sh[l]);
        Q[from[l]] += cimag(Sh[l]);
        P[to[l]] += creal(Sk[l]);
        Q[to[l]] += cimag(Sk[l]);
    }

    /* reduction step: partials onto the pre-built pattern (copy-add) */
    if (J) {
        int nnz = rp[nb];
        for (long e = 0; e < 4L * nnz; ++e) J[e] = 0.0;
        for (int i = 0; i < nb; ++i) {
            cplx ysh = (gs ? gs[i] : 0.0) + I * (bs ? bs[i] : 0.0);
            int kd = or_find(rp, ci, i, i);
            int dlen = rp[i + 1] - rp[i];
            int p = 2 * rp[i] + kd;
            cplx dv = 2.0 * vm[i] * conj(ysh);
            J[p + dlen] += creal(dv);
            J[2 * nnz + p + dlen] += cimag(dv);
        }
        for (int l = 0; l < nl; ++l) {
            if (skip && skip[l]) continue;
            int h = from[l], k = to[l];
            const cplx *q = dS + 8 * (long)l;
            /* (row bus, column bus, d/dtheta, d/dv) for the four slots */
            int rows[4] = {h, h, k, k}, cols[4] = {h, k, h, k};
            cplx dth[4] = {q[0], q[2], q[4], q[6]};
            cplx dvv[4] = {q[1], q[3], q[5], q[7]};
            for (int s = 0; s < 4; ++s) {
                int i = rows[s];
                int kpos = or_find(rp, ci, i, cols[s]);
                int dlen = rp[i + 1] - rp[i];
                int p = 2 * rp[i] + kpos;
                J[p] += creal(dth[s]);
                J[p + dlen] += creal(dvv[s]);
                J[2 * nnz + p] += cimag(dth[s]);
                J[2 * nnz + p + dlen] += cimag(dvv[s]);
            }
        }
    }
    free(Sh);
    free(Sk);
    free(dS);
    return nvalues;
}

/* ---------------------------------------------------- loss and adjoint --- */

/* L = sum_i wP_i (P_i - Ps_i)^2 + wQ_i (Q_i - Qs_i)^2 (summed in index order) */
double or_loss(int nb, const double *P, const double *Q, const double *Ps, const double *Qs,
               const double *wP, const double *wQ)
{
    double L = 0.0;
    for (int i = 0; i < nb; ++i) {
        double dp = P[i] - Ps[i], dq = Q[i] - Qs[i];
        L += wP[i] * dp * dp + wQ[i] * dq * dq;
    }
    return L;
}

/* State gradient of the loss through the assembled Jacobian:
   r_P = 2 wP (P - Ps), r_Q = 2 wQ (Q - Qs);
   dL/dtheta = J11^T r_P + J21^T r_Q,  dL/dv = J12^T r_P + J22^T r_Q. */
void or_adjoint_state(int nb, const int *rp, const int *ci, const double *J, const double *P,
                      const double *Q, const double *Ps, const double *Qs, const double *wP,
                      const double *wQ, double *gva, double *gvm)
{
    int nnz = rp[nb];
    for (int j = 0; j < nb; ++j) {
        gva[j] = 0.0;
        gvm[j] = 0.0;
    }
    for (int i = 0; i < nb; ++i) {
        double rP = 2.0 * wP[i] * (P[i] - Ps[i]);
        double rQ = 2.0 * wQ[i] * (Q[i] - Qs[i]);
        int d = rp[i + 1] - rp[i];
        for (int k = 0; k < d; ++k) {
            int j = ci[rp[i] + k];
            int p = 2 * rp[i] + k;
            gva[j] += J[p] * rP + J[2 * nnz + p] * rQ;
            gvm[j] += J[p + d] * rP + J[2 * nnz + p + d] * rQ;
        }
    }
}

/* loss contribution of buses h and k with branch l's parameters replaced by
   complex values (complex-step carrier); real-form injections. */
static cplx or_loss_pair_c(int nb, const int *rp, const int *ci, const double *yre, const double *yim,
                           const double *vm, const double *va, const double *Ps, const double *Qs,
                           const double *wP, const double *wQ, int h, int k, cplx dg, cplx db,
                           cplx dbsh, cplx dtap, double g0, double b0, double bsh0, double tap0,
                           double shift0)
{
    /* perturbed minus nominal stamps of branch l, in real form (G and B kept
       as complex carriers so the complex step passes through) */
    cplx g1 = g0 + dg, b1 = b0 + db, bsh1 = bsh0 + dbsh, m1 = tap0 + dtap;
    double c = cos(shift0), s = sin(shift0);
    /* G, B of the four stamps for parameters (g, b, bsh, m) */
    cplx Ghh1 = g1 / (m1 * m1), Bhh1 = (b1 + bsh1 / 2.0) / (m1 * m1);
    cplx Ghk1 = -(g1 * c - b1 * s) / m1, Bhk1 = -(g1 * s + b1 * c) / m1;
    cplx Gkh1 = -(g1 * c + b1 * s) / m1, Bkh1 = -(b1 * c - g1 * s) / m1;
    cplx Gkk1 = g1, Bkk1 = b1 + bsh1 / 2.0;
    double Ghh0 = g0 / (tap0 * tap0), Bhh0 = (b0 + bsh0 / 2.0) / (tap0 * tap0);
    double Ghk0 = -(g0 * c - b0 * s) / tap0, Bhk0 = -(g0 * s + b0 * c) / tap0;
    double Gkh0 = -(g0 * c + b0 * s) / tap0, Bkh0 = -(b0 * c - g0 * s) / tap0;
    double Gkk0 = g0, Bkk0 = b0 + bsh0 / 2.0;
    int rows[2] = {h, k};
    cplx L = 0.0;
    for (int t = 0; t < 2; ++t) {
        int i = rows[t];
        cplx p = 0.0, q = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int j = ci[e];
            cplx G = yre[e], B = yim[e];
            if (i == h && j == h) { G += Ghh1 - Ghh0; B += Bhh1 - Bhh0; }
            if (i == h && j == k) { G += Ghk1 - Ghk0; B += Bhk1 - Bhk0; }
            if (i == k && j == h) { G += Gkh1 - Gkh0; B += Bkh1 - Bkh0; }
            if (i == k && j == k) { G += Gkk1 - Gkk0; B += Bkk1 - Bkk0; }
            double d = va[i] - va[j];
            p += vm[j] * (G * cos(d) + B * sin(d));
            q += vm[j] * (G * sin(d) - B * cos(d));
        }
        cplx Pi = vm[i] * p, Qi = vm[i] * q;
        cplx dp = Pi - Ps[i], dq = Qi - Qs[i];
        L += wP[i] * dp * dp + wQ[i] * dq * dq;
    }
    return L;
}

/*
 * Branch-parameter gradient of the loss, dL/d(g, b, b_sh, tap) per branch, by
 * complex step through the real-form injections of the two terminal buses
 * (the only loss terms a branch parameter reaches).  The Ybus (rp, ci, yre,
 * yim) must be the one built from the same parameters.  Parallel branches are
 * handled because each branch's own stamps are perturbed, not the merged entry.
 */
void or_adjoint_params_cstep(int nb, int nl, const int *from, const int *to, const double *g,
                             const double *b, const double *bsh, const double *tap, const double *shift,
                             const int *rp, const int *ci, const double *yre, const double *yim,
                             const double *vm, const double *va, const double *Ps, const double *Qs,
                             const double *wP, const double *wQ, double *gg, double *gb, double *gbsh,
                             double *gtap)
{
    const double h = 1e-30;
    for (int l = 0; l < nl; ++l) {
        int hb = from[l], kb = to[l];
        cplx z = 0.0, st = I * h;
        gg[l] = cimag(or_loss_pair_c(nb, rp, ci, yre, yim, vm, va, Ps, Qs, wP, wQ, hb, kb, st, z, z, z,
                                     g[l], b[l], bsh[l], tap[l], shift[l])) / h;
        gb[l] = cimag(or_loss_pair_c(nb, rp, ci, yre, yim, vm, va, Ps, Qs, wP, wQ, hb, kb, z, st, z, z,
                                     g[l], b[l], bsh[l], tap[l], shift[l])) / h;
        gbsh[l] = cimag(or_loss_pair_c(nb, rp, ci, yre, yim, vm, va, Ps, Qs, wP, wQ, hb, kb, z, z, st, z,
                                       g[l], b[l], bsh[l], tap[l], shift[l])) / h;
        gtap[l] = cimag(or_loss_pair_c(nb, rp, ci, yre, yim, vm, va, Ps, Qs, wP, wQ, hb, kb, z, z, z, st,
                                       g[l], b[l], bsh[l], tap[l], shift[l])) / h;
    }
}

/* local loss (buses listed in bus[0..nbus)) with one coordinate offset by dx,
   in long double straight from the branch list (Eqs. 5-6 split into real and
   imaginary parts, bus shunt added), independent of the Ybus code paths */
static long double or_local_loss_ld(const int *from, const int *to, const double *g, const double *b,
                                    const double *bsh, const double *tap, const double *shift,
                                    const double *gs, const double *bs, const double *vm, const double *va,
                                    const double *Ps, const double *Qs, const double *wP, const double *wQ,
                                    const int *inc_ptr, const int *inc_br, const int *bus, int nbus,
                                    int kind, int idx, long double dx)
{
    long double L = 0.0L;
    for (int q = 0; q < nbus; ++q) {
        int i = bus[q];
        long double vi = vm[i] + ((kind == 1 && idx == i) ? dx : 0.0L);
        long double Pi = vi * vi * (gs ? gs[i] : 0.0), Qi = -vi * vi * (bs ? bs[i] : 0.0);
        for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; ++e) {
            int l = inc_br[e];
            int h = from[l], k = to[l];
            long double gl = g[l] + ((kind == 2 && idx == l) ? dx : 0.0L);
            long double bl = b[l] + ((kind == 3 && idx == l) ? dx : 0.0L);
            long double sl = bsh[l] + ((kind == 4 && idx == l) ? dx : 0.0L);
            long double ml = tap[l] + ((kind == 5 && idx == l) ? dx : 0.0L);
            long double vh = vm[h] + ((kind == 1 && idx == h) ? dx : 0.0L);
            long double vk = vm[k] + ((kind == 1 && idx == k) ? dx : 0.0L);
            long double th = va[h] + ((kind == 0 && idx == h) ? dx : 0.0L);
            long double tk = va[k] + ((kind == 0 && idx == k) ? dx : 0.0L);
            long double a = th - tk - shift[l];
            long double ca = cosl(a), sa = sinl(a);
            if (i == h) {
                Pi += vh * vh * gl / (ml * ml) - vh * vk / ml * (gl * ca + bl * sa);
                Qi += -vh * vh * (bl + sl / 2.0L) / (ml * ml) - vh * vk / ml * (gl * sa - bl * ca);
            } else {
                Pi += vk * vk * gl - vh * vk / ml * (gl * ca - bl * sa);
                Qi += -vk * vk * (bl + sl / 2.0L) - vh * vk / ml * (-gl * sa - bl * ca);
            }
        }
        long double dp = Pi - Ps[i], dq = Qi - Qs[i];
        L += wP[i] * dp * dp + wQ[i] * dq * dq;
    }
    return L;
}

/*
 * Central finite differences of the loss, (L(x+h) - L(x-h)) / 2h, for a batch
 * of coordinates, in long double, evaluating only the buses each coordinate
 * reaches.  kinds[c]: 0 theta_j, 1 v_j (idx = bus j); 2..5 g, b, b_sh, tap of
 * branch idx.  This is the independent, truncation-limited check of the
 * adjoint (about 1e-10 relative for h = 1e-7 on these grids).
 * Returns 0, or -1 on allocation failure.
 */
int or_loss_central_diff(int nb, int nl, const int *from, const int *to, const double *g, const double *b,
                         const double *bsh, const double *tap, const double *shift, const double *gs,
                         const double *bs, const double *vm, const double *va, const double *Ps,
                         const double *Qs, const double *wP, const double *wQ, int ncoord,
                         const int *kinds, const int *idxs, double step, double *out)
{
    int *inc_ptr = (int *)calloc((size_t)nb + 1, sizeof(int));
    int *inc_br = (int *)malloc(sizeof(int) * (size_t)(2 * nl + 1));
    int *fill = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    int *bus = (int *)malloc(sizeof(int) * (size_t)(2 * nl + 2));
    if (!inc_ptr || !inc_br || !fill || !bus) {
        free(inc_ptr);
        free(inc_br);
        free(fill);
        free(bus);
        return -1;
    }
    for (int l = 0; l < nl; ++l) {
        inc_ptr[from[l] + 1]++;
        inc_ptr[to[l] + 1]++;
    }
    for (int i = 0; i < nb; ++i) inc_ptr[i + 1] += inc_ptr[i];
    for (int i = 0; i < nb; ++i) fill[i] = inc_ptr[i];
    for (int l = 0; l < nl; ++l) {
        inc_br[fill[from[l]]++] = l;
        inc_br[fill[to[l]]++] = l;
    }
    for (int c = 0; c < ncoord; ++c) {
        int kind = kinds[c], idx = idxs[c], nbus = 0;
        if (kind <= 1) {
            bus[nbus++] = idx;
            for (int e = inc_ptr[idx]; e < inc_ptr[idx + 1]; ++e) {
                int l = inc_br[e];
                int o = from[l] == idx ? to[l] : from[l];
                int dup = 0;
                for (int r = 0; r < nbus; ++r)
                    if (bus[r] == o) dup = 1;
                if (!dup) bus[nbus++] = o;
            }
        } else {
            bus[nbus++] = from[idx];
            bus[nbus++] = to[idx];
        }
        long double hp = or_local_loss_ld(from, to, g, b, bsh, tap, shift, gs, bs, vm, va, Ps, Qs, wP, wQ,
                                          inc_ptr, inc_br, bus, nbus, kind, idx, (long double)step);
        long double hm = or_local_loss_ld(from, to, g, b, bsh, tap, shift, gs, bs, vm, va, Ps, Qs, wP, wQ,
                                          inc_ptr, inc_br, bus, nbus, kind, idx, -(long double)step);
        out[c] = (double)((hp - hm) / (2.0L * (long double)step));
    }
    free(inc_ptr);
    free(inc_br);
    free(fill);
    free(bus);
    return 0;
}
