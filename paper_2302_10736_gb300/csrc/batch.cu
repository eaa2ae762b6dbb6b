// batch.cu - C ABI of scenario batches: N-1 contingency evaluation and the
// adjoint of the mismatch loss (see k_batched.cu for the kernels).
#include <algorithm>
#include <climits>
#include <new>

#include "fastmath.cuh"
#include "pf_internal.h"

using namespace pf;

namespace pf {

// Outage metadata of branch l on the grid's sorted-terminal structure.
static ScenOut scen_outage(const HostTopo &H, int l)
{
    ScenOut o{-1, -1, -1, -1, 0, 0, 0, -1};
    if (l < 0) return o;
    const int th = 2 * l, tk = 2 * l + 1;
    o.l = l;
    o.h = H.owner(th);
    o.k = H.owner(tk);
    o.ph = H.tpos[th];
    o.pk = H.tpos[tk];
    o.kh = H.tkpos[th];
    o.kk = H.tkpos[tk];
    // the entry pair disappears unless another terminal of h runs to k
    int run = 0;
    for (int p = H.tp[o.h]; p < H.tp[o.h + 1]; ++p) run += H.tnbr[p].x == o.k;
    o.del = run == 1 ? 1 : 0;
    return o;
}

}  // namespace pf

namespace pf {

// The window plan of a batch: windows of at most tb buses and tfac x tb
// terminals (tfac = 0: the largest of 3, 2, 1 at which four CTAs of the
// batched Jacobian kernel share an SM's shared memory - its register budget
// allows four; with three, barrier and load stalls leave more of the FP64
// pipe idle: 1.53 against 1.47 ms for 1,024 N-1 scenarios of the 10,000-bus
// grid - else the largest at which one fits).  When the batch has fewer
// (scenario, window) items than the GPU has SMs, the windows are cut at equal
// cost into about one item per SM (more CTAs would only make the grid
// barriers dearer) and the adjoint keeps each item on one CTA (ghost).
pf_status batch_plan(const Grid *g, int nscen, int tb, int tfac, HostEw &E, bool &ghost)
{
    int dev = 0, nsm = 0, smem_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return set_error(PF_ECUDA, "batch: cannot query the device");
    auto smem_of = [](const HostEw &L) {
        return ew_smem_plan(L.max_nbus, L.max_nt, L.max_L, true).total + kTrigSmem;
    };
    const size_t kCtaReserve = 1024;   // shared memory the runtime keeps per resident CTA
    bool have = false;
    for (int tf = tfac ? tfac : 3; tf >= (tfac ? tfac : 1); --tf) {
        HostEw F;
        if (pf_status hs = host_ew(g->topo, tb, F, tf)) return hs;
        const size_t sm = smem_of(F);
        if (sm > kMaxSmem) continue;
        const bool four = 4 * (sm + kCtaReserve) <= (size_t)smem_sm;
        if (!have || four) {
            E = std::move(F);
            have = true;
        }
        if (four) break;
    }
    if (!have) return set_error(PF_EUNSUPPORTED, "batch: a window of %d buses / %d terminals per thread exceeds "
                                "shared memory", tb, tfac);
    ghost = false;
    if (nscen > 0 && (long long)nscen * E.nwin < nsm) {
        HostEw F;
        const int target = (nsm + nscen - 1) / nscen;
        if (host_ew(g->topo, tb, F, E.tfac, target) == PF_OK && F.nwin > E.nwin && smem_of(F) <= kMaxSmem)
            E = std::move(F);
        // latency-bound: the adjoint keeps each item on one CTA (k_adj1), which
        // forms its window's phasors itself (with its ghost buses) instead of a
        // separate phase and grid barrier
        ghost = adj1_smem_plan(E.max_nbus, E.max_nt, E.max_nph).total <= kMaxSmem;
    }
#ifdef PF_SELFCHECK
    if (pf_status hs = host_selfcheck(g->topo, E)) return hs;
#endif
    return PF_OK;
}

// Upload a window plan, replacing the batch's previous one (synchronizes st).
pf_status batch_upload(Batch *b, HostEw &E, bool ghost, cudaStream_t st)
{
    const Grid *g = b->g;
    // the small-batch adjoint's per-window branch lists; their counts ride in
    // the otherwise unused desc[2w+1].w
    std::vector<int2> brl;
    int max_nbr = 0;
    if (ghost) {
        std::vector<int> nbr;
        if (pf_status hs = host_window_branches(g->topo, E, brl, nbr, max_nbr)) return hs;
        for (int w = 0; w < E.nwin; ++w) E.desc[2 * w + 1].w = nbr[w];
    }
    cudaError_t e = cudaStreamSynchronize(st);   // no launch in flight still reads the old plan
    if (e != cudaSuccess) return cuda_error(e, "batch layout");
    for (void *p : {(void *)b->win_bus, (void *)b->rorder, (void *)b->desc, (void *)b->slotbus, (void *)b->tloc,
                    (void *)b->brl, (void *)b->lpart})
        b->arena.release(p);
    b->win_bus = b->rorder = b->slotbus = nullptr;
    b->desc = nullptr;
    b->tloc = b->brl = nullptr;
    b->lpart = nullptr;
    const size_t nw = (size_t)std::max(b->S, 1) * std::max(E.nwin, 1);
    if ((e = b->arena.alloc(&b->win_bus, E.win_bus.size())) ||
        (e = cudaMemcpyAsync(b->win_bus, E.win_bus.data(), sizeof(int) * E.win_bus.size(), cudaMemcpyHostToDevice,
                             st)) ||
        (e = b->arena.alloc(&b->rorder, E.rorder.size())) ||
        (e = cudaMemcpyAsync(b->rorder, E.rorder.data(), sizeof(int) * E.rorder.size(), cudaMemcpyHostToDevice,
                             st)) ||
        (ghost && ((e = b->arena.alloc(&b->desc, E.desc.size())) || (e = b->arena.alloc(&b->slotbus, E.slotbus.size())) ||
                   (e = b->arena.alloc(&b->tloc, E.tloc.size())) ||
                   (e = cudaMemcpyAsync(b->desc, E.desc.data(), sizeof(int4) * E.desc.size(), cudaMemcpyHostToDevice,
                                        st)) ||
                   (e = cudaMemcpyAsync(b->slotbus, E.slotbus.data(), sizeof(int) * E.slotbus.size(),
                                        cudaMemcpyHostToDevice, st)) ||
                   (e = cudaMemcpyAsync(b->tloc, E.tloc.data(), sizeof(int2) * E.tloc.size(), cudaMemcpyHostToDevice,
                                        st)) ||
                   (e = b->arena.alloc(&b->brl, std::max<size_t>(brl.size(), 1))) ||
                   (!brl.empty() &&
                    (e = cudaMemcpyAsync(b->brl, brl.data(), sizeof(int2) * brl.size(), cudaMemcpyHostToDevice, st))))) ||
        (e = b->arena.alloc(&b->lpart, nw)) || (e = cudaStreamSynchronize(st)))
        return cuda_error(e, "batch layout");
    b->tb = E.tb;
    b->tfac = E.tfac;
    b->nwin = E.nwin;
    b->max_L = E.max_L;
    b->max_nt = E.max_nt;
    b->max_nbus = E.max_nbus;
    b->ghost = ghost ? 1 : 0;
    b->max_nph = E.max_nph;
    b->max_nbr = max_nbr;
    for (int &r : b->resident) r = 0;   // shared memory and CTA counts change with the plan
    return PF_OK;
}

}  // namespace pf

PF_API pf_status batch_create(pf_grid *grid, int32_t nscen, const int32_t *outage, pf_stream stream, pf_batch **out)
{
    if (!out) return set_error(PF_EINVAL, "batch_create: out is NULL");
    *out = nullptr;
    if (!grid) return set_error(PF_EINVAL, "batch_create: grid is NULL");
    if (nscen < 0) return set_error(PF_EINVAL, "batch_create: nscen = %d", nscen);
    Grid *g = &grid->g;
    if ((long long)nscen * g->nb > (1LL << 40)) return set_error(PF_EUNSUPPORTED, "batch_create: batch too large");
    for (int s = 0; outage && s < nscen; ++s)
        if (outage[s] < -1 || outage[s] >= g->nl)
            return set_error(PF_EINVAL, "batch_create: outage[%d] = %d outside [-1, %d)", s, outage[s], g->nl);
    pf_batch *pb = new (std::nothrow) pf_batch;
    if (!pb) return set_error(PF_ENOMEM, "batch_create: host allocation failed");
    Batch *b = &pb->b;
    b->g = g;
    b->S = nscen;
    b->h_sc.resize(nscen);
    b->h_joff.assign(nscen + 1, 0);
    for (int s = 0; s < nscen; ++s) {
        b->h_sc[s] = scen_outage(g->topo, outage ? outage[s] : -1);
        b->h_joff[s + 1] = b->h_joff[s] + 4LL * (g->nnz - 2 * b->h_sc[s].del);
        b->has_outage |= b->h_sc[s].l >= 0;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete pb;
        return set_error(PF_ECUDA, "batch_create: cannot query the device");
    }
    b->cfg.window = 256;
    b->cfg.terminals_per_thread = 0;   // chosen by batch_plan
    b->cfg.ctas_per_sm = 0;
    b->cfg.adjoint_form = 0;
    b->cfg.ybus_lanes = g->cfg.ybus_lanes;
    b->cfg.ybus_block = g->cfg.ybus_block;
    cudaStream_t st = (cudaStream_t)stream;
    HostEw E;
    bool ghost = false;
    pf_status hs = batch_plan(g, nscen, b->cfg.window, 0, E, ghost);
    if (hs == PF_OK) hs = batch_upload(b, E, ghost, st);
    if (hs != PF_OK) {
        b->arena.free_all();
        delete pb;
        return hs;
    }
    b->cfg.terminals_per_thread = b->tfac;
    const size_t n = (size_t)nscen * g->nb;
    cudaError_t e = cudaSuccess;
    if ((e = b->arena.alloc(&b->sc, std::max(nscen, 1))) || (e = b->arena.alloc(&b->joff, nscen + 1)) ||
        (e = b->arena.alloc(&b->U, n)) || (e = b->arena.alloc(&b->V, n)) || (e = b->arena.alloc(&b->r, n)) ||
        (e = b->arena.alloc(&b->lscen, std::max(nscen, 1))) ||
        (nscen && (e = cudaMemcpyAsync(b->sc, b->h_sc.data(), sizeof(ScenOut) * nscen, cudaMemcpyHostToDevice, st))) ||
        (e = cudaMemcpyAsync(b->joff, b->h_joff.data(), sizeof(long long) * (nscen + 1), cudaMemcpyHostToDevice,
                             st)) ||
        (e = cudaStreamSynchronize(st))) {
        b->arena.free_all();
        delete pb;
        return cuda_error(e, "batch_create");
    }
    // a tuned configuration for this GPU and size class, if a cache file holds one
    if ((hs = batch_apply_cached(b, st)) != PF_OK) {
        b->arena.free_all();
        delete pb;
        return hs;
    }
    *out = pb;
    return PF_OK;
}

PF_API void batch_destroy(pf_batch *batch)
{
    if (!batch) return;
    batch->b.arena.free_all();
    delete batch;
}

PF_API pf_status batch_info(const pf_batch *batch, int32_t *nscen, int64_t *nnzJ_total)
{
    if (!batch) return set_error(PF_EINVAL, "batch_info: batch is NULL");
    if (nscen) *nscen = batch->b.S;
    if (nnzJ_total) *nnzJ_total = batch->b.h_joff.back();
    return PF_OK;
}

PF_API pf_status batch_jac_offsets(const pf_batch *batch, const int64_t **offsets)
{
    if (!batch || !offsets) return set_error(PF_EINVAL, "batch_jac_offsets: NULL argument");
    *offsets = reinterpret_cast<const int64_t *>(batch->b.joff);
    return PF_OK;
}

PF_API pf_status batch_jac_pattern(const pf_batch *batch, int32_t s, int32_t *rowptr, int32_t *colidx,
                                   int32_t *nnzJ_s)
{
    if (!batch) return set_error(PF_EINVAL, "batch_jac_pattern: batch is NULL");
    const Batch *b = &batch->b;
    if (s < 0 || s >= b->S) return set_error(PF_EINVAL, "batch_jac_pattern: scenario %d outside [0, %d)", s, b->S);
    const HostTopo &H = b->g->topo;
    const ScenOut &o = b->h_sc[s];
    const int nb = H.nb;
    // the scenario's Ybus pattern: the base rows without the removed pair
    std::vector<int> rps(nb + 1, 0), cis;
    cis.reserve(H.ci.size());
    for (int i = 0; i < nb; ++i) {
        for (int e = H.rp[i]; e < H.rp[i + 1]; ++e) {
            const int j = H.ci[e];
            if (o.del && ((i == o.h && j == o.k) || (i == o.k && j == o.h))) continue;
            cis.push_back(j);
        }
        rps[i + 1] = (int)cis.size();
    }
    const int nnz = rps[nb];
    if (nnzJ_s) *nnzJ_s = 4 * nnz;
    if (rowptr) {
        for (int blk = 0; blk < 2; ++blk)
            for (int i = 0; i < nb; ++i) rowptr[blk * nb + i] = 2 * nnz * blk + 2 * rps[i];
        rowptr[2 * nb] = 4 * nnz;
    }
    if (colidx) {
        for (int blk = 0; blk < 2; ++blk)
            for (int i = 0; i < nb; ++i) {
                const int d = rps[i + 1] - rps[i], base = 2 * nnz * blk + 2 * rps[i];
                for (int k = 0; k < d; ++k) {
                    colidx[base + k] = cis[rps[i] + k];
                    colidx[base + d + k] = nb + cis[rps[i] + k];
                }
            }
    }
    return PF_OK;
}

static pf_status check_batch(pf_batch *batch, const void *vm, const void *va, const char *name)
{
    if (!batch) return set_error(PF_EINVAL, "%s: batch is NULL", name);
    if (batch->b.S > 0 && batch->b.g->nb > 0 && (!vm || !va)) return set_error(PF_EINVAL, "%s: vm or va is NULL", name);
    return PF_OK;
}

PF_API pf_status inj_elementwise_batched(pf_batch *batch, const double *vm, const double *va, double *P, double *Q,
                                         pf_stream stream)
{
    pf_status st = check_batch(batch, vm, va, "inj_elementwise_batched");
    if (st) return st;
    if (batch->b.S == 0 || batch->b.g->nb == 0) return PF_OK;
    if (!P || !Q) return set_error(PF_EINVAL, "inj_elementwise_batched: P or Q is NULL");
    TraceScope t(batch->b.g, PF_K_INJ_EW_BATCHED, (cudaStream_t)stream);
    PF_CUDA(launch_ew_batched(&batch->b, false, vm, va, P, Q, nullptr, (cudaStream_t)stream));
    return PF_OK;
}

PF_API pf_status jac_elementwise_batched(pf_batch *batch, const double *vm, const double *va, double *P, double *Q,
                                         double *J, pf_stream stream)
{
    pf_status st = check_batch(batch, vm, va, "jac_elementwise_batched");
    if (st) return st;
    if (batch->b.S == 0 || batch->b.g->nb == 0) return PF_OK;
    if (!J) return set_error(PF_EINVAL, "jac_elementwise_batched: J is NULL");
    if ((P == nullptr) != (Q == nullptr))
        return set_error(PF_EINVAL, "jac_elementwise_batched: P and Q must both be set or both NULL");
    TraceScope t(batch->b.g, PF_K_JAC_EW_BATCHED, (cudaStream_t)stream);
    PF_CUDA(launch_ew_batched(&batch->b, true, vm, va, P, Q, J, (cudaStream_t)stream));
    return PF_OK;
}

static pf_status check_ybus_batch(pf_batch *batch, const char *name)
{
    if ((long long)batch->b.S * batch->b.g->nb > INT32_MAX)
        return set_error(PF_EUNSUPPORTED, "%s: nscen * nb above 2^31 - 1", name);
    return PF_OK;
}

PF_API pf_status inj_ybus_batched(pf_batch *batch, const double *vm, const double *va, double *P, double *Q,
                                  pf_stream stream)
{
    pf_status st = check_batch(batch, vm, va, "inj_ybus_batched");
    if (st) return st;
    if (batch->b.S == 0 || batch->b.g->nb == 0) return PF_OK;
    if (!P || !Q) return set_error(PF_EINVAL, "inj_ybus_batched: P or Q is NULL");
    if ((st = check_ybus_batch(batch, "inj_ybus_batched"))) return st;
    TraceScope t(batch->b.g, PF_K_INJ_YBUS_BATCHED, (cudaStream_t)stream);
    PF_CUDA(launch_ybus_batched(&batch->b, false, vm, va, P, Q, nullptr, (cudaStream_t)stream));
    return PF_OK;
}

PF_API pf_status jac_ybus_batched(pf_batch *batch, const double *vm, const double *va, double *P, double *Q,
                                  double *J, pf_stream stream)
{
    pf_status st = check_batch(batch, vm, va, "jac_ybus_batched");
    if (st) return st;
    if (batch->b.S == 0 || batch->b.g->nb == 0) return PF_OK;
    if (!J) return set_error(PF_EINVAL, "jac_ybus_batched: J is NULL");
    if ((P == nullptr) != (Q == nullptr))
        return set_error(PF_EINVAL, "jac_ybus_batched: P and Q must both be set or both NULL");
    if ((st = check_ybus_batch(batch, "jac_ybus_batched"))) return st;
    TraceScope t(batch->b.g, PF_K_JAC_YBUS_BATCHED, (cudaStream_t)stream);
    PF_CUDA(launch_ybus_batched(&batch->b, true, vm, va, P, Q, J, (cudaStream_t)stream));
    return PF_OK;
}

PF_API pf_status adjoint_elementwise(pf_batch *batch, const double *vm, const double *va, const double *Pspec,
                                     const double *Qspec, const double *wP, const double *wQ, const double *Lbar,
                                     double *L, double *Ltot, double *gvm, double *gva, double *gg, double *gb,
                                     double *gbsh, double *gtap, pf_stream stream)
{
    pf_status st = check_batch(batch, vm, va, "adjoint_elementwise");
    if (st) return st;
    if (batch->b.S == 0 || batch->b.g->nb == 0) return PF_OK;
    if (!Pspec || !Qspec || !wP || !wQ || !gvm || !gva)
        return set_error(PF_EINVAL, "adjoint_elementwise: a required array is NULL");
    const bool any = gg || gb || gbsh || gtap;
    if (any && !(gg && gb && gbsh && gtap))
        return set_error(PF_EINVAL, "adjoint_elementwise: gg, gb, gbsh, gtap must all be set or all NULL");
    TraceScope t(batch->b.g, PF_K_ADJOINT, (cudaStream_t)stream);
    PF_CUDA(launch_adjoint(&batch->b, vm, va, Pspec, Qspec, wP, wQ, Lbar, L, Ltot, gvm, gva, any ? gg : nullptr, gb,
                           gbsh, gtap, (cudaStream_t)stream));
    return PF_OK;
}

PF_API pf_status loss_elementwise(pf_batch *batch, const double *vm, const double *va, const double *Pspec,
                                  const double *Qspec, const double *wP, const double *wQ, double *L, double *Ltot,
                                  pf_stream stream)
{
    pf_status st = check_batch(batch, vm, va, "loss_elementwise");
    if (st) return st;
    if (batch->b.S == 0 || batch->b.g->nb == 0) return PF_OK;
    if (!Pspec || !Qspec || !wP || !wQ) return set_error(PF_EINVAL, "loss_elementwise: a required array is NULL");
    if (!L && !Ltot) return set_error(PF_EINVAL, "loss_elementwise: L and Ltot are both NULL");
    TraceScope t(batch->b.g, PF_K_LOSS, (cudaStream_t)stream);
    PF_CUDA(launch_loss(&batch->b, vm, va, Pspec, Qspec, wP, wQ, L, Ltot, (cudaStream_t)stream));
    return PF_OK;
}
