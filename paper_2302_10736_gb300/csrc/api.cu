// api.cu - C ABI entry points, validation and host-side structure build.
//
// Structure built once per topology (Sec. IV-A data structures, Alg. 2):
//   * sorted terminals: every branch has two terminals (t = 2l at h = from,
//     t = 2l+1 at k = to); they are ordered by (owner bus, other bus, branch)
//     so that a bus's terminals, and the parallel runs among them, are
//     contiguous - the terminal-to-bus and terminal-to-slot permutations of
//     the element-wise reduction;
//   * the Ybus CSR pattern and, per nonzero, the range of sorted terminals
//     whose stamps it sums (deterministic value assembly on the device);
//   * the canonical J pattern (closed form of Alg. 2);
//   * the element-wise windows of consecutive buses, cut at equal cost, with
//     their ghost buses and fixed-stride descriptors (host_layout.cpp).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>

#include "fastmath.cuh"
#include "pf_internal.h"

namespace pf {

static thread_local std::string g_last_error;

pf_status set_error(pf_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

std::atomic<int> g_alloc_countdown{-1};

// One process-wide maximum per (device, kernel): the attribute is a property
// of the kernel on a device, shared by every grid and batch, so it is only
// ever raised.  Lowering it for a smaller grid would make a larger grid's
// next launch fail.
cudaError_t ensure_dyn_smem(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = set[std::make_pair(dev, kernel)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

pf_status cuda_error(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();   // so that a later launch check does not see this failure
        return set_error(PF_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(PF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void DevArena::release(void *p)
{
    if (!p) return;
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it != ptrs.end()) {
        cudaFree(p);
        ptrs.erase(it);
    }
}

void DevArena::free_all()
{
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
}

template <class T>
static pf_status upload(DevArena &a, T **dst, const std::vector<T> &src, cudaStream_t s)
{
    PF_CUDA(a.alloc(dst, src.size()));
    if (!src.empty()) PF_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return PF_OK;
}

static bool finite_all(const double *x, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

static pf_status validate(const pf_grid_desc *d)
{
    if (!d) return set_error(PF_EINVAL, "ybus_build: desc is NULL");
    if (d->nb < 0 || d->nl < 0) return set_error(PF_EINVAL, "ybus_build: negative size nb=%d nl=%d", d->nb, d->nl);
    // 4 * nnzY must fit int32 (nnzY <= nb + 2 nl)
    if ((int64_t)d->nb + 2 * (int64_t)d->nl > (int64_t)(INT32_MAX / 4) - 64)
        return set_error(PF_EUNSUPPORTED, "ybus_build: nb + 2 nl = %lld exceeds the int32 Jacobian index range",
                         (long long)d->nb + 2 * (long long)d->nl);
    if (d->nl > 0 && (!d->from || !d->to || !d->g || !d->b || !d->bsh || !d->tap || !d->shift))
        return set_error(PF_EINVAL, "ybus_build: a branch array is NULL");
    for (int l = 0; l < d->nl; ++l) {
        int h = d->from[l], k = d->to[l];
        if (h < 0 || h >= d->nb || k < 0 || k >= d->nb)
            return set_error(PF_ETOPO, "ybus_build: branch %d joins bus %d and %d, outside [0, %d)", l, h, k, d->nb);
        if (h == k) return set_error(PF_ETOPO, "ybus_build: branch %d is a self loop at bus %d", l, h);
        if (!(d->tap[l] > 0.0) || !std::isfinite(d->tap[l]))
            return set_error(PF_EINVAL, "ybus_build: branch %d has tap %g (must be finite and > 0)", l, d->tap[l]);
    }
    if (d->nl > 0 && !(finite_all(d->g, d->nl) && finite_all(d->b, d->nl) && finite_all(d->bsh, d->nl) &&
                       finite_all(d->shift, d->nl)))
        return set_error(PF_EINVAL, "ybus_build: a branch parameter is not finite");
    if ((d->gs && !finite_all(d->gs, d->nb)) || (d->bs && !finite_all(d->bs, d->nb)))
        return set_error(PF_EINVAL, "ybus_build: a bus shunt is not finite");
    return PF_OK;
}

// Upload the topology structures (built on the host by host_topology).
static pf_status upload_topology(Grid *g, cudaStream_t s)
{
    const HostTopo &H = g->topo;
    const int nb = g->nb, T = 2 * g->nl;
    DevArena &a = g->arena;
    pf_status st;
    if ((st = upload(a, &g->rp, H.rp, s))) return st;
    if ((st = upload(a, &g->ci, H.ci, s))) return st;
    if ((st = upload(a, &g->ybeg, H.ybeg, s))) return st;
    if ((st = upload(a, &g->yend, H.yend, s))) return st;
    if ((st = upload(a, &g->ydiag, H.ydiag, s))) return st;
    if ((st = upload(a, &g->tpos, H.tpos, s))) return st;
    if ((st = upload(a, &g->tp, H.tp, s))) return st;
    if ((st = upload(a, &g->kd, H.kd, s))) return st;
    {
        std::vector<int> yrow(nb);
        for (int c0 = 0; c0 < nb; c0 += kYbusRowChunk) {
            const int c1 = std::min(nb, c0 + kYbusRowChunk);
            for (int i = c0; i < c1; ++i) yrow[i] = i;
            std::stable_sort(yrow.begin() + c0, yrow.begin() + c1,
                             [&](int x, int y) { return H.rp[x + 1] - H.rp[x] > H.rp[y + 1] - H.rp[y]; });
        }
        if ((st = upload(a, &g->yrow, yrow, s))) return st;
    }
    if ((st = upload(a, &g->tnbr, H.tnbr, s))) return st;
    if ((st = upload(a, &g->town, H.town, s))) return st;
    if ((st = upload(a, &g->tmir, H.tmir, s))) return st;
    {
        std::vector<int2> hk(g->nl);
        for (int l = 0; l < g->nl; ++l) hk[l] = make_int2(H.from[l], H.to[l]);
        if ((st = upload(a, &g->br_hk, hk, s))) return st;
        PF_CUDA(cudaStreamSynchronize(s));   // hk is freed on return
    }
    const size_t nl = (size_t)g->nl;
    PF_CUDA(a.alloc(&g->p_g, nl));
    PF_CUDA(a.alloc(&g->p_b, nl));
    PF_CUDA(a.alloc(&g->p_bsh, nl));
    PF_CUDA(a.alloc(&g->p_tap, nl));
    PF_CUDA(a.alloc(&g->p_shift, nl));
    PF_CUDA(a.alloc(&g->bus_yd, (size_t)nb));
    if ((st = upload(a, &g->jrp, H.jrp, s))) return st;
    if ((st = upload(a, &g->jci, H.jci, s))) return st;
    PF_CUDA(a.alloc(&g->yv, (size_t)g->nnz));
    PF_CUDA(a.alloc(&g->yfx, (size_t)g->nnz));
    PF_CUDA(a.alloc(&g->yce, (size_t)g->nnz));
    PF_CUDA(a.alloc(&g->tself, (size_t)T));
    PF_CUDA(a.alloc(&g->tcoup, (size_t)T));
    PF_CUDA(a.alloc(&g->tcfx, (size_t)T));
    PF_CUDA(a.alloc(&g->tce, (size_t)T));
    PF_CUDA(a.alloc(&g->br_aux, (size_t)g->nl));
    PF_CUDA(a.alloc(&g->bus_ysh, (size_t)nb));
    PF_CUDA(a.alloc(&g->ph_u, (size_t)nb));
    PF_CUDA(a.alloc(&g->ph_v, (size_t)nb));
    PF_CUDA(a.alloc(&g->err, 1));
    PF_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    PF_CUDA(a.alloc(&g->bar, kBarWords));
    PF_CUDA(cudaMemsetAsync(g->bar, 0, kBarWords * sizeof(unsigned int), s));
    PF_CUDA(cudaStreamSynchronize(s));  // host vectors stay alive, but keep setup ordered
    return PF_OK;
}

// Build (host), check and upload the element-wise windows for CTAs of `tb`
// threads (at most tb buses and tb terminals per window).  The windows are cut
// at equal estimated cost into a whole number of waves of the CTAs that fit
// on the GPU at once, so that every SM gets the same work.
static pf_status ew_fits(const HostEw &E, size_t *smem)
{
    const EwSmem plan = ew_smem_plan(E.max_nbus, E.max_nt, E.max_L, true, E.max_nph);
    *smem = plan.total + kTrigSmem;
    if (*smem > kMaxSmem)
        return set_error(PF_EUNSUPPORTED, "an element-wise window needs %u bytes of shared memory (max %u): a bus "
                                          "has too many branches for this library", (unsigned)*smem, kMaxSmem);
    return PF_OK;
}

static pf_status build_ew_layout(Grid *g, int tb, cudaStream_t s)
{
    HostEw E;
    size_t smem = 0;
    pf_status st = host_ew(g->topo, tb, E);
    if (st || (st = ew_fits(E, &smem))) return st;
    int dev = 0, nsm = 0, per_sm = 0;
    PF_CUDA(cudaGetDevice(&dev));
    PF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    PF_CUDA(ew_blocks_per_sm(tb, smem, &per_sm));
    for (int pass = 0; pass < 2 && per_sm > 0 && E.nwin > 1; ++pass) {
        const long long wave = (long long)nsm * per_sm;
        const int target = (int)std::min<long long>(wave * ((E.nwin + wave - 1) / wave), INT32_MAX);
        HostEw B;
        size_t smem_b = 0;
        if ((st = host_ew(g->topo, tb, B, 1, target)) || (st = ew_fits(B, &smem_b))) return st;
        int per_sm_b = 0;
        PF_CUDA(ew_blocks_per_sm(tb, smem_b, &per_sm_b));
        E = std::move(B);
        if (per_sm_b >= per_sm) break;   // the balanced windows still fit as planned
        per_sm = per_sm_b;               // fewer fit: balance again for the smaller wave
    }
#ifdef PF_SELFCHECK
    if ((st = host_selfcheck(g->topo, E))) return st;
#endif
    g->arena.release(g->ew.desc);
    g->arena.release(g->ew.slotbus);
    g->arena.release(g->ew.bmeta);
    g->arena.release(g->ew.rorder);
    g->arena.release(g->ew.tloc);
    g->ew = EwDev{};
    if ((st = upload(g->arena, &g->ew.desc, E.desc, s)) || (st = upload(g->arena, &g->ew.slotbus, E.slotbus, s)) ||
        (st = upload(g->arena, &g->ew.bmeta, E.bmeta, s)) || (st = upload(g->arena, &g->ew.rorder, E.rorder, s)) ||
        (st = upload(g->arena, &g->ew.tloc, E.tloc, s)))
        return st;
    g->ew.tb = E.tb;
    g->ew.nwin = E.nwin;
    g->ew.max_L = E.max_L;
    g->ew.max_nt = E.max_nt;
    g->ew.max_nbus = E.max_nbus;
    g->ew.max_nph = E.max_nph;
    PF_CUDA(cudaStreamSynchronize(s));  // E's vectors are freed on return
    return PF_OK;
}

pf_status refresh_values(Grid *g, const double *gg, const double *gb, const double *gbsh, const double *gtap,
                         const double *gshift, const double *gs, const double *bs, cudaStream_t s)
{
    PF_CUDA(launch_branch_constants(g, gg, gb, gbsh, gtap, gshift, s));
    PF_CUDA(launch_ybus_values(g, gs, bs, s));
    const size_t bytes = (size_t)g->nl * sizeof(double);
    if (bytes) {
        PF_CUDA(cudaMemcpyAsync(g->p_g, gg, bytes, cudaMemcpyDeviceToDevice, s));
        PF_CUDA(cudaMemcpyAsync(g->p_b, gb, bytes, cudaMemcpyDeviceToDevice, s));
        PF_CUDA(cudaMemcpyAsync(g->p_bsh, gbsh, bytes, cudaMemcpyDeviceToDevice, s));
        PF_CUDA(cudaMemcpyAsync(g->p_tap, gtap, bytes, cudaMemcpyDeviceToDevice, s));
        PF_CUDA(cudaMemcpyAsync(g->p_shift, gshift, bytes, cudaMemcpyDeviceToDevice, s));
    }
    return PF_OK;
}

static pf_status check_eval(pf_grid *grid, const void *vm, const void *va, const char *name)
{
    if (!grid) return set_error(PF_EINVAL, "%s: grid is NULL", name);
    if (grid->g.nb > 0 && (!vm || !va)) return set_error(PF_EINVAL, "%s: vm or va is NULL", name);
    return PF_OK;
}

}  // namespace pf

using namespace pf;

// ================================================================= ABI ====

PF_API const char *pf_status_str(pf_status s)
{
    switch (s) {
    case PF_OK: return "PF_OK";
    case PF_EINVAL: return "PF_EINVAL";
    case PF_ENOMEM: return "PF_ENOMEM";
    case PF_ECUDA: return "PF_ECUDA";
    case PF_ETOPO: return "PF_ETOPO";
    case PF_EDEVICE: return "PF_EDEVICE";
    case PF_ETIMEOUT: return "PF_ETIMEOUT";
    case PF_EUNSUPPORTED: return "PF_EUNSUPPORTED";
    case PF_ENOCONV: return "PF_ENOCONV";
    default: return "PF_UNKNOWN";
    }
}

PF_API const char *pf_last_error(void) { return g_last_error.c_str(); }

PF_API pf_status pf_debug_fail_allocations(int32_t after)
{
    if (after < -1) return set_error(PF_EINVAL, "pf_debug_fail_allocations: after = %d", after);
    g_alloc_countdown.store(after);
    return PF_OK;
}

PF_API pf_status ybus_build(const pf_grid_desc *d, pf_stream stream, pf_grid **out)
{
    if (!out) return set_error(PF_EINVAL, "ybus_build: out is NULL");
    *out = nullptr;
    pf_status st = validate(d);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    pf_grid *pg = new (std::nothrow) pf_grid;
    if (!pg) return set_error(PF_ENOMEM, "ybus_build: host allocation failed");
    Grid *g = &pg->g;
    g->nb = d->nb;
    g->nl = d->nl;
    g->cfg.ybus_lanes = 4;
    g->cfg.ybus_block = 256;
    g->cfg.ew_window = 256;
    g->cfg.ybus_fused = 1;
    if ((st = host_topology(d->nb, d->nl, d->from, d->to, g->topo))) {
        delete pg;
        return st;
    }
    g->nnz = g->topo.nnz;
    double *p[7] = {nullptr};
    const double *src[7] = {d->g, d->b, d->bsh, d->tap, d->shift, d->gs, d->bs};
    size_t len[7] = {(size_t)d->nl, (size_t)d->nl, (size_t)d->nl, (size_t)d->nl, (size_t)d->nl, (size_t)d->nb,
                     (size_t)d->nb};
    try {
        cudaError_t te = ensure_trig_table();
        if (te != cudaSuccess) throw cuda_error(te, "ybus_build: trig table");
        if ((st = upload_topology(g, s))) throw st;
        if ((st = build_ew_layout(g, g->cfg.ew_window, s))) throw st;
        for (int q = 0; q < 7; ++q) {
            if (!src[q]) continue;
            cudaError_t e = cudaMalloc(&p[q], std::max<size_t>(len[q], 1) * sizeof(double));
            if (e != cudaSuccess) throw cuda_error(e, "ybus_build: cudaMalloc(params)");
            e = cudaMemcpyAsync(p[q], src[q], len[q] * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) throw cuda_error(e, "ybus_build: cudaMemcpyAsync(params)");
        }
        if ((st = refresh_values(g, p[0], p[1], p[2], p[3], p[4], p[5], p[6], s))) throw st;
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) throw cuda_error(e, "ybus_build: cudaStreamSynchronize");
    } catch (pf_status err) {
        for (double *q : p) cudaFree(q);
        g->arena.free_all();
        delete pg;
        return err;
    }
    for (double *q : p) cudaFree(q);
    *out = pg;
    return PF_OK;
}

static void trace_free(Grid *g)
{
    for (cudaEvent_t e : g->tr_ev) cudaEventDestroy(e);
    g->tr_ev.clear();
    g->tr_kernel.clear();
    g->tr_n = 0;
}

PF_API void grid_destroy(pf_grid *grid)
{
    if (!grid) return;
    trace_free(&grid->g);
    grid->g.arena.free_all();
    delete grid;
}

PF_API pf_status grid_info(const pf_grid *grid, int32_t *nb, int32_t *nl, int32_t *nnzY)
{
    if (!grid) return set_error(PF_EINVAL, "grid_info: grid is NULL");
    if (nb) *nb = grid->g.nb;
    if (nl) *nl = grid->g.nl;
    if (nnzY) *nnzY = grid->g.nnz;
    return PF_OK;
}

PF_API pf_status grid_ew_windows(const pf_grid *grid, int32_t *out, int32_t max_windows, int32_t *nwin)
{
    if (!grid) return set_error(PF_EINVAL, "grid_ew_windows: grid is NULL");
    const Grid *g = &grid->g;
    const int n = g->ew.nwin;
    if (nwin) *nwin = n;
    if (!out || max_windows <= 0 || n == 0) return PF_OK;
    const int m = n < max_windows ? n : max_windows;
    std::vector<int4> d(2 * (size_t)m);
    PF_CUDA(cudaMemcpy(d.data(), g->ew.desc, d.size() * sizeof(int4), cudaMemcpyDeviceToHost));
    for (int w = 0; w < m; ++w) {
        int32_t *o = out + 5 * (size_t)w;
        o[0] = d[2 * w].x;
        o[1] = d[2 * w].y;
        o[2] = d[2 * w].z;
        o[3] = d[2 * w].w;
        o[4] = d[2 * w + 1].z;
    }
    return PF_OK;
}

PF_API pf_status grid_set_params(pf_grid *grid, const double *g_, const double *b_, const double *bsh_,
                                 const double *tap_, const double *shift_, const double *gs_, const double *bs_,
                                 pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "grid_set_params: grid is NULL");
    if (grid->g.nl > 0 && (!g_ || !b_ || !bsh_ || !tap_ || !shift_))
        return set_error(PF_EINVAL, "grid_set_params: a branch parameter array is NULL");
    return refresh_values(&grid->g, g_, b_, bsh_, tap_, shift_, gs_, bs_, (cudaStream_t)stream);
}

PF_API pf_status ybus_get(const pf_grid *grid, int32_t *nnz, const int32_t **rowptr, const int32_t **colidx,
                          const double **values)
{
    if (!grid) return set_error(PF_EINVAL, "ybus_get: grid is NULL");
    if (nnz) *nnz = grid->g.nnz;
    if (rowptr) *rowptr = grid->g.rp;
    if (colidx) *colidx = grid->g.ci;
    if (values) *values = reinterpret_cast<const double *>(grid->g.yv);
    return PF_OK;
}

PF_API pf_status jac_pattern(const pf_grid *grid, int32_t *nnzJ, const int32_t **rowptr, const int32_t **colidx)
{
    if (!grid) return set_error(PF_EINVAL, "jac_pattern: grid is NULL");
    if (nnzJ) *nnzJ = 4 * grid->g.nnz;
    if (rowptr) *rowptr = grid->g.jrp;
    if (colidx) *colidx = grid->g.jci;
    return PF_OK;
}

PF_API pf_status inj_ybus(pf_grid *grid, const double *vm, const double *va, double *P, double *Q, pf_stream stream)
{
    pf_status st = check_eval(grid, vm, va, "inj_ybus");
    if (st) return st;
    Grid *g = &grid->g;
    if (g->nb == 0) return PF_OK;
    if (!P || !Q) return set_error(PF_EINVAL, "inj_ybus: P or Q is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (g->cfg.ybus_fused) {   // one launch: the phasors formed inside the row kernel
        TraceScope t(g, PF_K_INJ_YBUS, s);
        PF_CUDA(launch_ybus_fused(g, false, vm, va, P, Q, nullptr, s));
        return PF_OK;
    }
    {
        TraceScope t(g, PF_K_PHASOR, s);
        PF_CUDA(launch_phasor_fix(g->nb, vm, va, g->ph_u, s));
    }
    {
        TraceScope t(g, PF_K_INJ_YBUS, s);
        PF_CUDA(launch_ybus_rows(g, 1, false, nullptr, nullptr, g->ph_u, false, P, Q, nullptr, g->cfg.ybus_lanes,
                                 g->cfg.ybus_block, s));
    }
    return PF_OK;
}

PF_API pf_status inj_elementwise(pf_grid *grid, const double *vm, const double *va, double *P, double *Q,
                                 pf_stream stream)
{
    pf_status st = check_eval(grid, vm, va, "inj_elementwise");
    if (st) return st;
    Grid *g = &grid->g;
    if (g->nb == 0) return PF_OK;
    if (!P || !Q) return set_error(PF_EINVAL, "inj_elementwise: P or Q is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    {
        TraceScope t(g, PF_K_INJ_EW, s);
        PF_CUDA(launch_inj_ew(g, vm, va, P, Q, s));
    }
    return PF_OK;
}

PF_API pf_status jac_ybus(pf_grid *grid, const double *vm, const double *va, double *P, double *Q, double *J,
                          pf_stream stream)
{
    pf_status st = check_eval(grid, vm, va, "jac_ybus");
    if (st) return st;
    Grid *g = &grid->g;
    if (g->nb == 0) return PF_OK;
    if (!J) return set_error(PF_EINVAL, "jac_ybus: J is NULL");
    if ((P == nullptr) != (Q == nullptr)) return set_error(PF_EINVAL, "jac_ybus: P and Q must both be set or both NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (g->cfg.ybus_fused) {   // one launch: the phasors formed inside the row kernel
        TraceScope t(g, PF_K_JAC_YBUS, s);
        PF_CUDA(launch_ybus_fused(g, true, vm, va, P, Q, J, s));
        return PF_OK;
    }
    {
        TraceScope t(g, PF_K_PHASOR, s);
        PF_CUDA(launch_phasor_fix(g->nb, vm, va, g->ph_u, s));
    }
    {
        TraceScope t(g, PF_K_JAC_YBUS, s);
        PF_CUDA(launch_ybus_rows(g, 1, false, nullptr, nullptr, g->ph_u, true, P, Q, J, g->cfg.ybus_lanes,
                                 g->cfg.ybus_block, s));
    }
    return PF_OK;
}

PF_API pf_status jac_elementwise(pf_grid *grid, const double *vm, const double *va, double *P, double *Q, double *J,
                                 pf_stream stream)
{
    pf_status st = check_eval(grid, vm, va, "jac_elementwise");
    if (st) return st;
    Grid *g = &grid->g;
    if (g->nb == 0) return PF_OK;
    if (!J) return set_error(PF_EINVAL, "jac_elementwise: J is NULL");
    if ((P == nullptr) != (Q == nullptr))
        return set_error(PF_EINVAL, "jac_elementwise: P and Q must both be set or both NULL");
    cudaStream_t s = (cudaStream_t)stream;
    {
        TraceScope t(g, PF_K_JAC_EW, s);
        PF_CUDA(launch_jac_ew(g, vm, va, P, Q, J, s));
    }
    return PF_OK;
}

// Device address of a host buffer that kernels can write directly
// (page-locked and mapped: cudaHostAlloc, cudaHostRegister), else nullptr.
static void *mapped_device_ptr(const void *h)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// eval_host and eval_host_async: `sync` says whether the call waits for the
// results; the asynchronous form takes page-locked buffers only.
static pf_status eval_host_impl(pf_grid *grid, int32_t method, const double *vm, const double *va, double *P,
                                double *Q, double *J, pf_stream stream, bool sync, const char *name)
{
    pf_status st = check_eval(grid, vm, va, name);
    if (st) return st;
    if (method != 0 && method != 1) return set_error(PF_EINVAL, "%s: method must be 0 (Ybus) or 1 (element-wise)", name);
    Grid *g = &grid->g;
    if (g->nb == 0) return PF_OK;
    if (!P || !Q || !J) return set_error(PF_EINVAL, "%s: P, Q and J must be non-NULL", name);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = (size_t)g->nb, nJ = 4 * (size_t)g->nnz;
    void *dvm = mapped_device_ptr(vm), *dva = mapped_device_ptr(va);
    void *dP = mapped_device_ptr(P), *dQ = mapped_device_ptr(Q), *dJ = mapped_device_ptr(J);
    if (!sync && !(dvm && dva && dP && dQ && dJ))
        return set_error(PF_EINVAL, "%s: vm, va, P, Q and J must all be page-locked host buffers", name);
    if (!g->st_J) {
        double **const out[5] = {&g->st_vm, &g->st_va, &g->st_P, &g->st_Q, &g->st_J};
        const size_t n[5] = {nb, nb, nb, nb, nJ};
        PF_CUDA(alloc_all(g->arena, out, n));
    }
    if (method == 1 && dP && dQ && dJ) {
        // page-locked, mapped host buffers: the kernel reads vm, va and stores
        // P, Q, J across the host link while it runs; no staging copies
        if (!dvm || !dva) {
            PF_CUDA(cudaMemcpyAsync(g->st_vm, vm, nb * 8, cudaMemcpyHostToDevice, s));
            PF_CUDA(cudaMemcpyAsync(g->st_va, va, nb * 8, cudaMemcpyHostToDevice, s));
            dvm = g->st_vm;
            dva = g->st_va;
        }
        {
            TraceScope t(g, PF_K_JAC_EW, s);
            PF_CUDA(launch_jac_ew(g, (const double *)dvm, (const double *)dva, (double *)dP, (double *)dQ,
                                  (double *)dJ, s, true));
        }
        if (sync) PF_CUDA(cudaStreamSynchronize(s));
        return PF_OK;
    }
    PF_CUDA(cudaMemcpyAsync(g->st_vm, vm, nb * 8, cudaMemcpyHostToDevice, s));
    PF_CUDA(cudaMemcpyAsync(g->st_va, va, nb * 8, cudaMemcpyHostToDevice, s));
    st = method == 0 ? jac_ybus(grid, g->st_vm, g->st_va, g->st_P, g->st_Q, g->st_J, stream)
                     : jac_elementwise(grid, g->st_vm, g->st_va, g->st_P, g->st_Q, g->st_J, stream);
    if (st) return st;
    PF_CUDA(cudaMemcpyAsync(P, g->st_P, nb * 8, cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaMemcpyAsync(Q, g->st_Q, nb * 8, cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaMemcpyAsync(J, g->st_J, nJ * 8, cudaMemcpyDeviceToHost, s));
    if (sync) PF_CUDA(cudaStreamSynchronize(s));
    return PF_OK;
}

PF_API pf_status eval_host(pf_grid *grid, int32_t method, const double *vm, const double *va, double *P, double *Q,
                           double *J, pf_stream stream)
{
    return eval_host_impl(grid, method, vm, va, P, Q, J, stream, true, "eval_host");
}

PF_API pf_status eval_host_async(pf_grid *grid, int32_t method, const double *vm, const double *va, double *P,
                                 double *Q, double *J, pf_stream stream)
{
    return eval_host_impl(grid, method, vm, va, P, Q, J, stream, false, "eval_host_async");
}

PF_API pf_status phasor(int32_t n, const double *vm, const double *va, double *U, double *V, pf_stream stream)
{
    if (n < 0) return set_error(PF_EINVAL, "phasor: n = %d", n);
    if (n == 0) return PF_OK;
    if (!vm || !va || !U || !V) return set_error(PF_EINVAL, "phasor: NULL pointer");
    if (((uintptr_t)U & 31u) || ((uintptr_t)V & 15u))
        return set_error(PF_EINVAL, "phasor: U must be 32-byte and V 16-byte aligned");
    PF_CUDA(ensure_trig_table());
    PF_CUDA(launch_phasor(n, vm, va, reinterpret_cast<double4_32a *>(U), reinterpret_cast<double2 *>(V),
                          (cudaStream_t)stream));
    return PF_OK;
}

PF_API pf_status grid_inject_barrier_fault(pf_grid *grid, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "grid_inject_barrier_fault: grid is NULL");
    // both arrival counters far below every target (as signed differences),
    // so the next batched launch's first barrier never completes
    const unsigned int phantom = 0x80000000u;
    cudaStream_t st = (cudaStream_t)stream;
    PF_CUDA(cudaMemcpyAsync(grid->g.bar + 32, &phantom, sizeof(phantom), cudaMemcpyHostToDevice, st));
    PF_CUDA(cudaMemcpyAsync(grid->g.bar + 64, &phantom, sizeof(phantom), cudaMemcpyHostToDevice, st));
    PF_CUDA(cudaStreamSynchronize(st));   // `phantom` is a stack variable
    return PF_OK;
}

PF_API pf_status grid_get_config(const pf_grid *grid, pf_config *cfg)
{
    if (!grid || !cfg) return set_error(PF_EINVAL, "grid_get_config: NULL argument");
    *cfg = grid->g.cfg;
    return PF_OK;
}

static bool valid_lanes(int w) { return w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32; }

PF_API pf_status grid_set_config(pf_grid *grid, const pf_config *cfg, pf_stream stream)
{
    if (!grid || !cfg) return set_error(PF_EINVAL, "grid_set_config: NULL argument");
    if (!valid_lanes(cfg->ybus_lanes)) return set_error(PF_EINVAL, "ybus_lanes must be 1, 2, 4, 8, 16 or 32");
    if (cfg->ybus_block < 32 || cfg->ybus_block > 512 || cfg->ybus_block % 32)
        return set_error(PF_EINVAL, "ybus_block must be a multiple of 32 in [32, 512]");
    if (cfg->ybus_fused != 0 && cfg->ybus_fused != 1) return set_error(PF_EINVAL, "ybus_fused must be 0 or 1");
    Grid *g = &grid->g;
    cudaStream_t s = (cudaStream_t)stream;
    if (cfg->ew_window != g->ew.tb) {
        pf_status st = build_ew_layout(g, cfg->ew_window, s);
        if (st) g->cfg.ew_window = g->ew.tb;
        if (st) return st;
        PF_CUDA(cudaStreamSynchronize(s));
    }
    g->cfg = *cfg;
    return PF_OK;
}

PF_API pf_status grid_check_error(pf_grid *grid, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "grid_check_error: grid is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    PF_CUDA(cudaMemcpyAsync(&h, grid->g.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
    if (h == DEV_OK) return PF_OK;
    PF_CUDA(cudaMemsetAsync(grid->g.err, 0, sizeof(int), s));
    // a kernel that gave up may have left the grid barrier half-way: start it afresh
    PF_CUDA(cudaMemsetAsync(grid->g.bar, 0, kBarWords * sizeof(unsigned int), s));
    PF_CUDA(cudaStreamSynchronize(s));
    if (h == DEV_TIMEOUT) return set_error(PF_ETIMEOUT, "a device-side wait gave up (error word %d)", h);
    if (h == DEV_SINGULAR)
        return set_error(PF_EDEVICE, "jac_reduced_solve met a zero or non-finite pivot (error word %d)", h);
    return set_error(PF_EDEVICE, "a kernel reported device error word %d", h);
}

// ---------------------------------------------------------- autotuner ----

static pf_status time_it(float *ms_out, int reps, cudaStream_t s, pf_status (*fn)(void *), void *ctx)
{
    cudaEvent_t e0, e1;
    PF_CUDA(cudaEventCreate(&e0));
    PF_CUDA(cudaEventCreate(&e1));
    pf_status st = PF_OK;
    for (int r = 0; r < 2 && !st; ++r) st = fn(ctx);
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && !st; ++r) st = fn(ctx);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (e != cudaSuccess) return cuda_error(e, "autotune: cudaEventSynchronize");
    *ms_out = ms / (float)reps;
    return PF_OK;
}

struct TuneCtx {
    pf_grid *grid;
    const double *vm, *va;
    double *P, *Q, *J;
    cudaStream_t s;
};

static pf_status run_jac_ybus(void *c)
{
    TuneCtx *t = (TuneCtx *)c;
    return jac_ybus(t->grid, t->vm, t->va, t->P, t->Q, t->J, t->s);
}

static pf_status run_jac_ew(void *c)
{
    TuneCtx *t = (TuneCtx *)c;
    return jac_elementwise(t->grid, t->vm, t->va, t->P, t->Q, t->J, t->s);
}

PF_API pf_status grid_autotune(pf_grid *grid, const double *vm, const double *va, int32_t reps, pf_stream stream,
                               pf_config *best)
{
    pf_status st = check_eval(grid, vm, va, "grid_autotune");
    if (st) return st;
    Grid *g = &grid->g;
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->nb == 0) {
        if (best) *best = g->cfg;
        return PF_OK;
    }
    TuneCtx ctx{grid, vm, va, nullptr, nullptr, nullptr, s};
    PF_CUDA(cudaMalloc(&ctx.P, (size_t)g->nb * 8));
    PF_CUDA(cudaMalloc(&ctx.Q, (size_t)g->nb * 8));
    PF_CUDA(cudaMalloc(&ctx.J, (size_t)4 * g->nnz * 8 + 8));
    pf_config cfg = g->cfg, keep = g->cfg;
    float best_y = 1e30f, best_e = 1e30f;
    const int lanes[] = {1, 2, 4, 8, 16, 32}, blocks[] = {128, 256, 512};
    for (int fused : {0, 1})
        for (int w : lanes)
            for (int bk : blocks) {
                g->cfg.ybus_fused = fused;
                g->cfg.ybus_lanes = w;
                g->cfg.ybus_block = bk;
                float ms;
                if ((st = time_it(&ms, reps, s, run_jac_ybus, &ctx))) goto out;
                if (ms < best_y) {
                    best_y = ms;
                    cfg.ybus_fused = fused;
                    cfg.ybus_lanes = w;
                    cfg.ybus_block = bk;
                }
            }
    g->cfg.ybus_fused = cfg.ybus_fused;
    g->cfg.ybus_lanes = cfg.ybus_lanes;
    g->cfg.ybus_block = cfg.ybus_block;
    for (int win : {128, 256}) {
        pf_config c2 = g->cfg;
        c2.ew_window = win;
        if ((st = grid_set_config(grid, &c2, stream))) {
            if (st == PF_EUNSUPPORTED) {  // window too large for shared memory on this grid
                st = PF_OK;
                continue;
            }
            goto out;
        }
        float ms;
        if ((st = time_it(&ms, reps, s, run_jac_ew, &ctx))) goto out;
        if (ms < best_e) {
            best_e = ms;
            cfg.ew_window = win;
        }
    }
    st = grid_set_config(grid, &cfg, stream);
out:
    if (st) g->cfg = keep;
    cudaFree(ctx.P);
    cudaFree(ctx.Q);
    cudaFree(ctx.J);
    if (!st && best) *best = g->cfg;
    return st;
}

// ------------------------------------------------------------- tracer ----

PF_API const char *pf_kernel_name(int32_t k)
{
    static const char *names[PF_K_COUNT] = {"phasor",         "inj_ybus",       "jac_ybus",        "inj_ew",
                                            "jac_ew",         "inj_ew_batched", "jac_ew_batched",  "adjoint",
                                            "inj_ybus_batched", "jac_ybus_batched", "reduce", "loss", "lu"};
    return (k >= 0 && k < PF_K_COUNT) ? names[k] : "?";
}

PF_API pf_status grid_trace_enable(pf_grid *grid, int32_t capacity)
{
    if (!grid) return set_error(PF_EINVAL, "grid_trace_enable: grid is NULL");
    if (capacity < 0 || capacity > (1 << 20)) return set_error(PF_EINVAL, "grid_trace_enable: capacity %d", capacity);
    Grid *g = &grid->g;
    trace_free(g);
    if (capacity == 0) return PF_OK;
    g->tr_ev.resize(2 * (size_t)capacity, nullptr);
    g->tr_kernel.assign(capacity, -1);
    for (auto &e : g->tr_ev) {
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) {
            e = nullptr;
            for (auto &f : g->tr_ev)
                if (f) cudaEventDestroy(f);
            g->tr_ev.clear();
            g->tr_kernel.clear();
            return cuda_error(err, "grid_trace_enable: cudaEventCreate");
        }
    }
    return PF_OK;
}

PF_API pf_status grid_trace_read(pf_grid *grid, pf_trace_rec *out, int32_t cap, int32_t *n)
{
    if (!grid || (!out && cap > 0) || !n) return set_error(PF_EINVAL, "grid_trace_read: NULL argument");
    Grid *g = &grid->g;
    int m = std::min(g->tr_n, (int)cap);
    for (int i = 0; i < m; ++i) {
        PF_CUDA(cudaEventSynchronize(g->tr_ev[2 * i + 1]));
        float ms = 0.f;
        PF_CUDA(cudaEventElapsedTime(&ms, g->tr_ev[2 * i], g->tr_ev[2 * i + 1]));
        out[i].kernel = g->tr_kernel[i];
        out[i].ms = ms;
    }
    *n = m;
    g->tr_n = 0;
    return PF_OK;
}

// ---------------------------------------------------------- self-check ----

PF_API pf_status grid_selfcheck(const pf_grid_desc *d, int32_t window, int32_t nwin_target)
{
    pf_status st = validate(d);
    if (st) return st;
    if (nwin_target < 0) return set_error(PF_EINVAL, "grid_selfcheck: nwin_target = %d", nwin_target);
    HostTopo H;
    HostEw E;
    if ((st = host_topology(d->nb, d->nl, d->from, d->to, H))) return st;
    if ((st = host_ew(H, window, E, 1, nwin_target))) return st;
    if ((st = host_selfcheck(H, E))) return st;
    // the small-batch adjoint's per-window branch lists (every branch once)
    std::vector<int2> brl;
    std::vector<int> nbr;
    int max_nbr = 0;
    return host_window_branches(H, E, brl, nbr, max_nbr);
}
