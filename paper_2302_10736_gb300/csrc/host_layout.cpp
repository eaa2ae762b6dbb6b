// host_layout.cpp - host-only construction of every index structure the
// kernels use, plus a self-check of the invariants their memory accesses rely
// on (run on the CPU by the tests, and in debug builds before upload).
//
//   sorted terminals   terminal t = 2l (h = from[l] end) or 2l+1 (k = to[l]
//                      end), ordered by (owner bus, other bus, branch): the
//                      terminal-to-bus permutation of the reduction (Eq. 7)
//   Ybus pattern       row i = {i} U {other bus of i's terminals}, sorted;
//                      parallel branches share an entry; per entry the range
//                      of sorted terminals whose stamps it sums
//   J pattern          closed form of Alg. 2 (see include/pfgrid.h)
//   element-wise       sliced-ELL by bus window (see EwLayout)
#include <algorithm>
#include <cstdint>

#include "pf_internal.h"

namespace pf {

pf_status host_topology(int nb, int nl, const int *from, const int *to, HostTopo &H)
{
    const int T = 2 * nl;
    H.nb = nb;
    H.nl = nl;
    H.from.assign(from, from + nl);
    H.to.assign(to, to + nl);
    H.tp.assign(nb + 1, 0);
    for (int t = 0; t < T; ++t) H.tp[H.owner(t) + 1]++;
    for (int i = 0; i < nb; ++i) H.tp[i + 1] += H.tp[i];
    H.tsort.assign(T, 0);
    {
        std::vector<int> fill(H.tp.begin(), H.tp.end() - 1);
        for (int t = 0; t < T; ++t) H.tsort[fill[H.owner(t)]++] = t;
    }
    for (int i = 0; i < nb; ++i) {
        std::sort(H.tsort.begin() + H.tp[i], H.tsort.begin() + H.tp[i + 1], [&](int a, int c) {
            int oa = H.other(a), oc = H.other(c);
            return oa != oc ? oa < oc : a < c;
        });
    }
    H.rp.assign(nb + 1, 0);
    H.ci.clear();
    H.ci.reserve((size_t)nb + T);
    H.ybeg.clear();
    H.yend.clear();
    H.ydiag.clear();
    H.kd.assign(nb, 0);
    H.tkpos.assign(T, 0);
    H.taccum.assign(T, 0);
    for (int i = 0; i < nb; ++i) {
        const int p0 = H.tp[i], p1 = H.tp[i + 1], row_start = (int)H.ci.size();
        bool diag_done = false;
        auto emit_diag = [&]() {
            H.kd[i] = (int)H.ci.size() - row_start;
            H.ci.push_back(i);
            H.ybeg.push_back(p0);
            H.yend.push_back(p1);
            H.ydiag.push_back(i);
            diag_done = true;
        };
        int p = p0;
        while (p < p1) {
            const int j = H.other(H.tsort[p]);
            if (!diag_done && j > i) emit_diag();
            int q = p;
            while (q < p1 && H.other(H.tsort[q]) == j) {
                const int t = H.tsort[q];
                H.tkpos[t] = (int)H.ci.size() - row_start;
                H.taccum[t] = q > p ? 1 : 0;
                ++q;
            }
            H.ci.push_back(j);
            H.ybeg.push_back(p);
            H.yend.push_back(q);
            H.ydiag.push_back(-1);
            p = q;
        }
        if (!diag_done) emit_diag();
        H.rp[i + 1] = (int)H.ci.size();
    }
    H.nnz = H.rp[nb];
    H.tpos.assign(T, 0);
    for (int p = 0; p < T; ++p) H.tpos[H.tsort[p]] = p;
    const int nnz = H.nnz;
    H.jrp.assign(2 * (size_t)nb + 1, 0);
    H.jci.assign(4 * (size_t)nnz, 0);
    for (int blk = 0; blk < 2; ++blk)
        for (int i = 0; i < nb; ++i) {
            const int d = H.rp[i + 1] - H.rp[i], base = 2 * nnz * blk + 2 * H.rp[i];
            H.jrp[blk * nb + i] = base;
            for (int k = 0; k < d; ++k) {
                H.jci[base + k] = H.ci[H.rp[i] + k];
                H.jci[base + d + k] = nb + H.ci[H.rp[i] + k];
            }
        }
    H.jrp[2 * (size_t)nb] = 4 * nnz;
    return PF_OK;
}

pf_status host_ew(const HostTopo &H, int window, HostEw &E)
{
    if (window != 64 && window != 128 && window != 256 && window != 512)
        return set_error(PF_EINVAL, "ew_window must be 64, 128, 256 or 512 (got %d)", window);
    const int nb = H.nb, T = 2 * H.nl;
    E = HostEw{};
    E.window = window;
    E.nwin = (nb + window - 1) / window;
    const int nslot = E.nwin * window, nwarp = nslot / 32;
    E.meta.assign(nslot, make_int4(-1, 0, 0, 0));
    E.kd.assign(nslot, 0);
    E.wmeta.assign(nwarp, make_int2(0, 0));
    E.term_ent.assign(T, 0);
    std::vector<int> order(window);
    long long nent = 0;
    for (int w = 0; w < E.nwin; ++w) {
        const int b0 = w * window, b1 = std::min(b0 + window, nb), n = b1 - b0;
        for (int r = 0; r < n; ++r) order[r] = b0 + r;
        std::stable_sort(order.begin(), order.begin() + n,
                         [&](int x, int y) { return (H.tp[x + 1] - H.tp[x]) > (H.tp[y + 1] - H.tp[y]); });
        E.max_L = std::max(E.max_L, 2 * (H.rp[b1] - H.rp[b0]));
        for (int r = 0; r < n; ++r) {
            const int bus = order[r];
            E.meta[w * window + r] =
                make_int4(bus, H.tp[bus + 1] - H.tp[bus], 2 * (H.rp[bus] - H.rp[b0]), H.rp[bus + 1] - H.rp[bus]);
            E.kd[w * window + r] = H.kd[bus];
        }
        for (int wi = 0; wi < window / 32; ++wi) {
            int mx = 0;
            for (int l = 0; l < 32; ++l) mx = std::max(mx, E.meta[w * window + wi * 32 + l].y);
            E.wmeta[w * (window / 32) + wi] = make_int2((int)nent, mx);
            nent += 32LL * mx;
        }
    }
    if (nent > INT32_MAX / 2) return set_error(PF_EUNSUPPORTED, "element-wise layout too large (%lld entries)", nent);
    E.nent = (int)nent;
    E.nbr.assign((size_t)nent, make_int2(0, 0));
    for (int sl = 0; sl < nslot; ++sl) {
        const int bus = E.meta[sl].x;
        if (bus < 0) continue;
        const int2 wm = E.wmeta[sl / 32];
        const int lane = sl % 32;
        for (int k = 0; k < E.meta[sl].y; ++k) {
            const int t = H.tsort[H.tp[bus] + k];
            const int e = wm.x + 32 * k + lane;
            E.term_ent[t] = e;
            E.nbr[e] = make_int2(H.other(t), H.tkpos[t] | (H.taccum[t] ? EW_ACCUM : 0));
        }
        for (int k = E.meta[sl].y; k < wm.y; ++k) E.nbr[wm.x + 32 * k + lane] = make_int2(bus, 0);
    }
    return PF_OK;
}

size_t ew_jac_smem_bytes(const HostEw &E) { return (size_t)(2 * E.max_L + 2 * E.window) * sizeof(double); }

#define CHECK(cond, ...)                                       \
    do {                                                       \
        if (!(cond)) return set_error(PF_EINVAL, __VA_ARGS__); \
    } while (0)

pf_status host_selfcheck(const HostTopo &H, const HostEw &E)
{
    const int nb = H.nb, nnz = H.nnz, T = 2 * H.nl;
    // Ybus CSR
    CHECK((int)H.rp.size() == nb + 1 && H.rp[0] == 0 && H.rp[nb] == nnz, "rowptr ends");
    CHECK((long long)nnz * 4 < INT32_MAX, "nnzJ exceeds int32");
    for (int i = 0; i < nb; ++i) {
        CHECK(H.rp[i + 1] > H.rp[i], "row %d empty (diagonal missing)", i);
        for (int e = H.rp[i]; e < H.rp[i + 1]; ++e) {
            CHECK(H.ci[e] >= 0 && H.ci[e] < nb, "colidx out of range at %d", e);
            if (e > H.rp[i]) CHECK(H.ci[e] > H.ci[e - 1], "row %d not strictly sorted", i);
            CHECK(H.ybeg[e] >= 0 && H.ybeg[e] <= H.yend[e] && H.yend[e] <= T, "stamp range at %d", e);
            CHECK(H.ydiag[e] == (H.ci[e] == i ? i : -1), "diag flag at %d", e);
        }
        CHECK(H.kd[i] >= 0 && H.kd[i] < H.rp[i + 1] - H.rp[i] && H.ci[H.rp[i] + H.kd[i]] == i, "diag pos %d", i);
    }
    for (int t = 0; t < T; ++t) {
        const int o = H.owner(t), q = H.other(t);
        CHECK(H.tkpos[t] >= 0 && H.tkpos[t] < H.rp[o + 1] - H.rp[o], "kpos range t=%d", t);
        CHECK(H.ci[H.rp[o] + H.tkpos[t]] == q, "kpos column t=%d", t);
        CHECK(H.tsort[H.tpos[t]] == t, "tpos inverse t=%d", t);
    }
    // element-wise layout: every access of k_jac_ew / k_inj_ew stays in bounds
    const int W = E.window, nslot = E.nwin * W;
    CHECK((int)E.meta.size() == nslot && (int)E.kd.size() == nslot && (int)E.wmeta.size() == nslot / 32,
          "slot array sizes");
    std::vector<int> seen_bus(nb, 0), seen_ent(E.nent, 0);
    for (int w = 0; w < E.nwin; ++w) {
        const int b0 = w * W, b1 = std::min(b0 + W, nb);
        const int L = 2 * (H.rp[b1] - H.rp[b0]);
        CHECK(L <= E.max_L, "window %d L > max_L", w);
        for (int r = 0; r < W; ++r) {
            const int sl = w * W + r;
            const int4 m = E.meta[sl];
            const int2 wm = E.wmeta[sl / 32];
            if (m.x < 0) {
                CHECK(r >= b1 - b0, "empty slot inside a full window %d", w);
                continue;
            }
            CHECK(m.x >= b0 && m.x < b1, "slot bus outside window");
            CHECK(++seen_bus[m.x] == 1, "bus %d in two slots", m.x);
            CHECK(m.y == H.tp[m.x + 1] - H.tp[m.x] && m.y <= wm.y, "terminal count slot %d", sl);
            CHECK(m.w == H.rp[m.x + 1] - H.rp[m.x], "row length slot %d", sl);
            CHECK(m.z >= 0 && m.z + 2 * m.w <= L, "row slice outside the window slice, slot %d", sl);
            CHECK(E.kd[sl] >= 0 && E.kd[sl] < m.w, "diag pos slot %d", sl);
            for (int k = 0; k < wm.y; ++k) {
                const long long e = (long long)wm.x + 32LL * k + (sl % 32);
                CHECK(e >= 0 && e < E.nent, "entry %lld outside [0, %d)", e, E.nent);
                const int2 nq = E.nbr[e];
                CHECK(nq.x >= 0 && nq.x < nb, "gather index out of range at entry %lld", e);
                if (k < m.y) {
                    CHECK(++seen_ent[e] == 1, "entry %lld used twice", e);
                    const int kp = nq.y & EW_KMASK;
                    CHECK(kp >= 0 && kp < m.w && kp != E.kd[sl], "kpos entry %lld", e);
                    CHECK(m.z + kp + m.w < L, "staging index entry %lld", e);
                }
            }
        }
    }
    for (int i = 0; i < nb; ++i) CHECK(seen_bus[i] == 1, "bus %d has no slot", i);
    for (int t = 0; t < T; ++t) {
        const int e = E.term_ent[t];
        CHECK(e >= 0 && e < E.nent && seen_ent[e] == 1, "terminal %d entry", t);
        CHECK(E.nbr[e].x == H.other(t), "terminal %d gather index", t);
    }
    CHECK(ew_jac_smem_bytes(E) <= 227 * 1024, "window needs %zu bytes of shared memory", ew_jac_smem_bytes(E));
    return PF_OK;
}

}  // namespace pf
