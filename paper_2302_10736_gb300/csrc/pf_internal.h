// pf_internal.h - internal structures of libpfgrid (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "pfgrid.h"

#define PF_API extern "C" __attribute__((visibility("default")))

namespace pf {

// --------------------------------------------------------------- errors --
pf_status set_error(pf_status s, const char *fmt, ...);
pf_status cuda_error(cudaError_t e, const char *what);
#define PF_CUDA(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return pf::cuda_error(e_, #call); \
    } while (0)

// device error word codes (written by kernels, read by grid_check_error)
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BADINDEX = 2 };

// ------------------------------------------------- device buffer owner --
struct DevArena {
    std::vector<void *> ptrs;
    template <class T>
    cudaError_t alloc(T **p, size_t n)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, n > 0 ? n * sizeof(T) : 16);
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            *p = static_cast<T *>(q);
        }
        return e;
    }
    void release(void *p);
    void free_all();
};

// ------------------------------------------------ host index structures --
// Topology-only structures, built once on the host (host_layout.cpp).
struct HostTopo {
    int nb = 0, nl = 0, nnz = 0;
    std::vector<int> from, to;
    std::vector<int> tp;        // [nb+1] terminals of bus i: tsort[tp[i] .. tp[i+1])
    std::vector<int> tsort;     // [2nl] terminal ids sorted by (owner, other, branch)
    std::vector<int> tpos;      // [2nl] sorted position of terminal t
    std::vector<int> tkpos;     // [2nl] position of the other bus in the owner's Ybus row
    std::vector<int> taccum;    // [2nl] 1 if not the first terminal of its (owner, other) run
    std::vector<int> rp, ci;    // Ybus CSR pattern
    std::vector<int> ybeg, yend, ydiag;  // per nnz: sorted-terminal stamp range; row if diagonal else -1
    std::vector<int> kd;        // [nb] position of the diagonal in row i
    std::vector<int> jrp, jci;  // canonical J pattern
    int owner(int t) const { return (t & 1) ? to[t >> 1] : from[t >> 1]; }
    int other(int t) const { return (t & 1) ? from[t >> 1] : to[t >> 1]; }
};

// Element-wise layout (sliced-ELL by bus window): one CTA per window of W
// buses, one bus per thread; inside a window buses are ordered by terminal
// count (descending) so the 32 lanes of a warp loop over equally many
// terminals; entry (warp, k, lane) lives at warp_ebase + 32 k + lane, so the
// k-th terminals of a warp's buses are read with coalesced loads.
struct HostEw {
    int window = 0, nwin = 0, nent = 0;
    int max_L = 0;                 // max over windows of 2 * (Ybus nnz of the window's rows)
    std::vector<int4> meta;        // [nwin*W] {bus or -1, terminal count, 2*(rp[bus]-rp[b0]), row length d}
    std::vector<int> kd;           // [nwin*W] diagonal position in the slot bus's row
    std::vector<int2> wmeta;       // [nwin*W/32] {entry base, max terminal count}
    std::vector<int2> nbr;         // [nent] {other bus, kpos | EW_ACCUM}
    std::vector<int> term_ent;     // [2nl] entry of terminal t
};
enum : int { EW_ACCUM = 0x40000000, EW_KMASK = 0x3fffffff };

pf_status host_topology(int nb, int nl, const int *from, const int *to, HostTopo &H);
pf_status host_ew(const HostTopo &H, int window, HostEw &E);
pf_status host_selfcheck(const HostTopo &H, const HostEw &E);
size_t ew_jac_smem_bytes(const HostEw &E);

// ------------------------------------------------ device-side structure --
struct EwDev {
    int window = 0, nwin = 0, nent = 0, max_L = 0;
    int4 *slot_meta = nullptr;
    int *slot_kd = nullptr;
    double2 *slot_ysh = nullptr;   // [nwin*W] bus shunt of the slot's bus
    int2 *warp_meta = nullptr;
    double2 *ent_ys = nullptr;     // [nent] self constant of the terminal
    double2 *ent_yc = nullptr;     // [nent] coupling constant of the terminal
    int2 *ent_nbr = nullptr;
    int *term_ent = nullptr;
};

struct Grid {
    int nb = 0, nl = 0, nnz = 0;
    pf_config cfg{};
    DevArena arena;
    HostTopo topo;
    // Ybus (device)
    int *rp = nullptr, *ci = nullptr;
    double2 *yv = nullptr;
    int *ybeg = nullptr, *yend = nullptr, *ydiag = nullptr;
    // J pattern (device)
    int *jrp = nullptr, *jci = nullptr;
    // terminal constants in sorted-terminal order (device)
    double2 *tself = nullptr, *tcoup = nullptr;
    int *tpos = nullptr;
    double2 *bus_ysh = nullptr;
    EwDev ew;
    // per-call workspace (device)
    double4_32a *ph_u = nullptr;   // [nb] {cos, sin, v, 1/v}
    double2 *ph_v = nullptr;       // [nb] V = v e^{j theta}
    int *err = nullptr;            // device error word
    // eval_host staging (lazy)
    double *st_vm = nullptr, *st_va = nullptr, *st_P = nullptr, *st_Q = nullptr, *st_J = nullptr;
    // tracer: events [2 * capacity], kernel id per record
    std::vector<cudaEvent_t> tr_ev;
    std::vector<int> tr_kernel;
    int tr_n = 0;
};

// Brackets one kernel launch with tracer events when tracing is on.
struct TraceScope {
    Grid *g;
    int slot;
    cudaStream_t s;
    TraceScope(Grid *g_, int kernel, cudaStream_t s_) : g(g_), slot(-1), s(s_)
    {
        if (!g->tr_ev.empty() && g->tr_n < (int)g->tr_kernel.size()) {
            slot = g->tr_n++;
            g->tr_kernel[slot] = kernel;
            cudaEventRecord(g->tr_ev[2 * slot], s);
        }
    }
    ~TraceScope()
    {
        if (slot >= 0) cudaEventRecord(g->tr_ev[2 * slot + 1], s);
    }
};

// kernel launchers (k_*.cu); each returns cudaGetLastError() of its launch(es)
cudaError_t launch_branch_constants(Grid *g, const double *gg, const double *gb, const double *gbsh,
                                    const double *gtap, const double *gshift, cudaStream_t s);
cudaError_t launch_ybus_values(Grid *g, const double *gs, const double *bs, cudaStream_t s);
cudaError_t launch_ew_scatter(Grid *g, cudaStream_t s);
cudaError_t launch_phasor_u(int nb, const double *vm, const double *va, double4_32a *out, cudaStream_t s);
cudaError_t launch_phasor_v(int nb, const double *vm, const double *va, double2 *out, cudaStream_t s);
cudaError_t launch_inj_ybus(const Grid *g, const double2 *V, double *P, double *Q, cudaStream_t s);
cudaError_t launch_jac_ybus(const Grid *g, const double4_32a *U, double *P, double *Q, double *J, cudaStream_t s);
cudaError_t launch_inj_ew_vm(const Grid *g, const double *vm, const double2 *V, double *P, double *Q, cudaStream_t s);
cudaError_t launch_jac_ew(const Grid *g, const double4_32a *U, double *P, double *Q, double *J, cudaStream_t s);

}  // namespace pf

struct pf_grid {
    pf::Grid g;
};
