// k_setup.cu - parameter-dependent setup kernels and the phasor step.
//
// Branch constants (Sec. IV-C.1: constants "calculated once ahead of time"):
// every terminal t of branch l gets a self constant Ys_t and a coupling
// constant Yc_t such that its complex power (Eqs. 5-6) is
//     S_t = v_o^2 conj(Ys_t) + conj(Yc_t) V_o conj(V_q)      (o owner, q other bus)
// with, for y_s = g + j b, y_h = y_k = j b_sh / 2 and tap m e^{j phi} at h:
//     h terminal: Ys = (y_s + y_h) / m^2,   Yc = -y_s e^{ j phi} / m
//     k terminal: Ys =  y_s + y_k,          Yc = -y_s e^{-j phi} / m
// The same constants are the pi-model stamps of the Ybus, so the Ybus value
// of (i, j) is the sum of the coupling constants of the terminals (i -> j)
// and the diagonal is the bus shunt plus the self constants of all terminals
// of bus i, summed in a fixed order (no atomics).
#include "pf_internal.h"

namespace pf {

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

__global__ void k_bus_shunt(int nb, const double *__restrict__ gs, const double *__restrict__ bs, double2 *ysh)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    ysh[i] = make_double2(gs ? gs[i] : 0.0, bs ? bs[i] : 0.0);
}

__global__ void k_branch_constants(int nl, const double *__restrict__ g, const double *__restrict__ b,
                                   const double *__restrict__ bsh, const double *__restrict__ tap,
                                   const double *__restrict__ shift, const int *__restrict__ tpos,
                                   double2 *__restrict__ tself, double2 *__restrict__ tcoup)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const double gl = g[l], bl = b[l], half = 0.5 * bsh[l];
    const double im = 1.0 / tap[l], im2 = im * im;
    double sp, cp;
    sincos(shift[l], &sp, &cp);
    const double2 ys_h = make_double2(gl * im2, (bl + half) * im2);
    const double2 ys_k = make_double2(gl, bl + half);
    // y_s e^{+j phi} and y_s e^{-j phi}
    const double ar = gl * cp - bl * sp, ai = gl * sp + bl * cp;
    const double br = gl * cp + bl * sp, bi = bl * cp - gl * sp;
    const int ph = tpos[2 * l], pk = tpos[2 * l + 1];
    tself[ph] = ys_h;
    tcoup[ph] = make_double2(-ar * im, -ai * im);
    tself[pk] = ys_k;
    tcoup[pk] = make_double2(-br * im, -bi * im);
}

__global__ void k_ybus_values(int nnz, const int *__restrict__ ybeg, const int *__restrict__ yend,
                              const int *__restrict__ ydiag, const double2 *__restrict__ tself,
                              const double2 *__restrict__ tcoup, const double2 *__restrict__ bus_ysh,
                              double2 *__restrict__ yv)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int d = ydiag[e];
    double2 acc = d >= 0 ? bus_ysh[d] : make_double2(0.0, 0.0);
    const double2 *src = d >= 0 ? tself : tcoup;
    for (int p = ybeg[e]; p < yend[e]; ++p) {
        const double2 c = src[p];
        acc.x += c.x;
        acc.y += c.y;
    }
    yv[e] = acc;
}

__global__ void k_ew_scatter(int T, const int *__restrict__ term_ent, const int *__restrict__ tpos,
                             const double2 *__restrict__ tself, const double2 *__restrict__ tcoup,
                             double2 *__restrict__ ent_ys, double2 *__restrict__ ent_yc)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int e = term_ent[t], p = tpos[t];
    ent_ys[e] = tself[p];
    ent_yc[e] = tcoup[p];
}

__global__ void k_ew_slot_ysh(int nslot, const int4 *__restrict__ meta, const double2 *__restrict__ bus_ysh,
                              double2 *__restrict__ slot_ysh)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslot) return;
    const int bus = meta[s].x;
    slot_ysh[s] = bus >= 0 ? bus_ysh[bus] : make_double2(0.0, 0.0);
}

// Phasor step (Sec. IV-B.1 step 1): U = e^{j theta}; stored with v and 1/v
// for the Jacobian kernels, or V = v U for the injection kernels.
__global__ void k_phasor_u(int nb, const double *__restrict__ vm, const double *__restrict__ va,
                           double4_32a *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double s, c;
    sincos(va[i], &s, &c);
    const double v = vm[i];
    out[i] = make_double4_32a(c, s, v, __drcp_rn(v));
}

__global__ void k_phasor_v(int nb, const double *__restrict__ vm, const double *__restrict__ va,
                           double2 *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double s, c;
    sincos(va[i], &s, &c);
    const double v = vm[i];
    out[i] = make_double2(v * c, v * s);
}

cudaError_t launch_branch_constants(Grid *g, const double *gg, const double *gb, const double *gbsh,
                                    const double *gtap, const double *gshift, cudaStream_t s)
{
    if (g->nl > 0)
        k_branch_constants<<<nblk(g->nl, 256), 256, 0, s>>>(g->nl, gg, gb, gbsh, gtap, gshift, g->tpos, g->tself,
                                                            g->tcoup);
    return cudaGetLastError();
}

cudaError_t launch_ybus_values(Grid *g, const double *gs, const double *bs, cudaStream_t s)
{
    if (g->nb > 0) k_bus_shunt<<<nblk(g->nb, 256), 256, 0, s>>>(g->nb, gs, bs, g->bus_ysh);
    if (g->nnz > 0)
        k_ybus_values<<<nblk(g->nnz, 256), 256, 0, s>>>(g->nnz, g->ybeg, g->yend, g->ydiag, g->tself, g->tcoup,
                                                        g->bus_ysh, g->yv);
    return cudaGetLastError();
}

cudaError_t launch_ew_scatter(Grid *g, cudaStream_t s)
{
    const int T = 2 * g->nl, nslot = g->ew.nwin * g->ew.window;
    if (T > 0)
        k_ew_scatter<<<nblk(T, 256), 256, 0, s>>>(T, g->ew.term_ent, g->tpos, g->tself, g->tcoup, g->ew.ent_ys,
                                                  g->ew.ent_yc);
    if (nslot > 0) k_ew_slot_ysh<<<nblk(nslot, 256), 256, 0, s>>>(nslot, g->ew.slot_meta, g->bus_ysh, g->ew.slot_ysh);
    return cudaGetLastError();
}

cudaError_t launch_phasor_u(int nb, const double *vm, const double *va, double4_32a *out, cudaStream_t s)
{
    if (nb > 0) k_phasor_u<<<nblk(nb, 256), 256, 0, s>>>(nb, vm, va, out);
    return cudaGetLastError();
}

cudaError_t launch_phasor_v(int nb, const double *vm, const double *va, double2 *out, cudaStream_t s)
{
    if (nb > 0) k_phasor_v<<<nblk(nb, 256), 256, 0, s>>>(nb, vm, va, out);
    return cudaGetLastError();
}

}  // namespace pf
