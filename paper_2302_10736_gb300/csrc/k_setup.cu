// k_setup.cu - parameter-dependent setup kernels and the phasor step.
//
// Branch constants (Sec. IV-C.1 precomputes them once per parameter set):
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
#include <mutex>
#include <vector>

#include "fastmath.cuh"
#include "fixrot.cuh"
#include "isincos.cuh"
#include "pf_internal.h"
#include "ptx.cuh"

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
                                   double2 *__restrict__ tself, double2 *__restrict__ tcoup,
                                   longlong2 *__restrict__ tcfx, int *__restrict__ tce,
                                   double4_32a *__restrict__ aux)
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
    // the coupling constants in the block floating point of the element-wise kernels
    int64_t fr, fi;
    tce[ph] = fix_block(-ar * im, -ai * im, &fr, &fi);
    tcfx[ph] = make_longlong2(fr, fi);
    tce[pk] = fix_block(-br * im, -bi * im, &fr, &fi);
    tcfx[pk] = make_longlong2(fr, fi);
    aux[l] = make_double4_32a(im, cp, sp, -(bl + half));   // for the parameter gradients of the adjoint
}

__global__ void k_ybus_values(int nnz, const int *__restrict__ ybeg, const int *__restrict__ yend,
                              const int *__restrict__ ydiag, const double2 *__restrict__ tself,
                              const double2 *__restrict__ tcoup, const double2 *__restrict__ bus_ysh,
                              double2 *__restrict__ yv, longlong2 *__restrict__ yfx, int *__restrict__ yce)
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
    int64_t fr, fi;
    yce[e] = fix_block(acc.x, acc.y, &fr, &fi);   // the fixed-point form of the Ybus kernels
    yfx[e] = make_longlong2(fr, fi);
}

// Per-bus self sum Yd = y_sh + sum of the self constants of the bus's
// terminals (sorted order): the parameter-only part of Eq. 7.
__global__ void k_bus_yd(int nb, const int *__restrict__ tp, const double2 *__restrict__ tself,
                         const double2 *__restrict__ bus_ysh, double2 *__restrict__ yd)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double2 acc = bus_ysh[i];
    for (int p = tp[i]; p < tp[i + 1]; ++p) {
        acc.x += tself[p].x;
        acc.y += tself[p].y;
    }
    yd[i] = acc;
}

// kITrigCopies copies of the first-quadrant (cos, sin) table of isincos.cuh:
// every CTA copies one into shared memory at its start, and the copies spread
// those reads over many L2 lines
__device__ ITrig g_itrig_tab[kITrigCopies * kITrigN];

// Phasor step (Sec. IV-B.1 step 1): U = e^{j theta} with v and 1/v (gathered
// by the Jacobian kernels) and V = v U (gathered by the injection kernels and
// by the element-wise Jacobian for the owner bus).  The sine and cosine run on
// the integer pipe (isincos.cuh); 6 FP64 instructions per bus (fast_rcp 4 +
// the hardware approximation, V 2).
__global__ void __launch_bounds__(256) k_phasor(int nb, const double *__restrict__ vm,
                                                const double *__restrict__ va, double4_32a *__restrict__ U,
                                                double2 *__restrict__ V)
{
    __shared__ ITrig tab[kITrigN];
    pdl_launch_dependents();   // the evaluation kernel may start loading its static data now
    if (threadIdx.x < kITrigN) tab[threadIdx.x] = g_itrig_tab[(blockIdx.x % kITrigCopies) * kITrigN + threadIdx.x];
    // launched as a programmatic dependent: the previous kernel in the stream
    // (which may read U and V, or write vm and va) has completed after this
    pdl_wait();
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double s, c;
    int_sincos(va[i], tab, &s, &c);
    const double v = vm[i];
    U[i] = make_double4_32a(c, s, v, fast_rcp(v));
    V[i] = make_double2(v * c, v * s);
}

// The phasor step in the fixed-point form of the batched Ybus kernels
// (fixrot.cuh): U = {2^62 cos, 2^62 sin (64-bit integers stored bit for bit),
// v, 0}; no FP64 instruction.
__global__ void __launch_bounds__(256) k_phasor_fix(int nb, const double *__restrict__ vm,
                                                    const double *__restrict__ va, double4_32a *__restrict__ U)
{
    __shared__ ITrig tab[kITrigN];
    pdl_launch_dependents();
    if (threadIdx.x < kITrigN) tab[threadIdx.x] = g_itrig_tab[(blockIdx.x % kITrigCopies) * kITrigN + threadIdx.x];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb) {   // the state: into L2 before the wait (no data returned), read after it
        prefetch_l2(va + i);
        prefetch_l2(vm + i);
    }
    pdl_wait();
    __syncthreads();
    if (i >= nb) return;
    int64_t c, s;
    int_sincos_q62(va[i], tab, &c, &s);
    U[i] = make_double4_32a(__longlong_as_double(c), __longlong_as_double(s), vm[i], 0.0);
}

// Upload the trig table once per device (synchronous, first use only).
static std::mutex g_trig_mu;
static const ITrig *g_trig_ptr[256] = {nullptr};

const ITrig *trig_table()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
    std::lock_guard<std::mutex> lk(g_trig_mu);
    return g_trig_ptr[dev];
}

cudaError_t ensure_trig_table()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_trig_mu);
    if (g_trig_ptr[dev]) return cudaSuccess;
    std::vector<ITrig> copies((size_t)kITrigCopies * kITrigN);
    for (int c = 0; c < kITrigCopies; ++c)
        for (int j = 0; j < kITrigN; ++j) copies[(size_t)c * kITrigN + j] = kITrigTable[j];
    if ((e = cudaMemcpyToSymbol(g_itrig_tab, copies.data(), copies.size() * sizeof(ITrig))) != cudaSuccess) return e;
    void *p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_itrig_tab)) != cudaSuccess) return e;
    g_trig_ptr[dev] = static_cast<const ITrig *>(p);
    return cudaSuccess;
}

cudaError_t launch_branch_constants(Grid *g, const double *gg, const double *gb, const double *gbsh,
                                    const double *gtap, const double *gshift, cudaStream_t s)
{
    if (g->nl > 0)
        k_branch_constants<<<nblk(g->nl, 256), 256, 0, s>>>(g->nl, gg, gb, gbsh, gtap, gshift, g->tpos, g->tself,
                                                            g->tcoup, g->tcfx, g->tce, g->br_aux);
    return cudaGetLastError();
}

cudaError_t launch_ybus_values(Grid *g, const double *gs, const double *bs, cudaStream_t s)
{
    if (g->nb > 0) k_bus_shunt<<<nblk(g->nb, 256), 256, 0, s>>>(g->nb, gs, bs, g->bus_ysh);
    if (g->nnz > 0)
        k_ybus_values<<<nblk(g->nnz, 256), 256, 0, s>>>(g->nnz, g->ybeg, g->yend, g->ydiag, g->tself, g->tcoup,
                                                        g->bus_ysh, g->yv, g->yfx, g->yce);
    if (g->nb > 0) k_bus_yd<<<nblk(g->nb, 256), 256, 0, s>>>(g->nb, g->tp, g->tself, g->bus_ysh, g->bus_yd);
    return cudaGetLastError();
}

cudaError_t launch_phasor_fix(int nb, const double *vm, const double *va, double4_32a *U, cudaStream_t s)
{
    if (nb > 0) return launch_k(k_phasor_fix, nblk(nb, 256), 256, 0, s, true, nb, vm, va, U);
    return cudaSuccess;
}

cudaError_t launch_phasor(int nb, const double *vm, const double *va, double4_32a *U, double2 *V, cudaStream_t s)
{
    if (nb > 0) return launch_k(k_phasor, nblk(nb, 256), 256, 0, s, true, nb, vm, va, U, V);
    return cudaSuccess;
}

}  // namespace pf
