// host_layout.cpp - host-only construction of every index structure the
// kernels use, plus a self-check of the invariants their memory accesses rely
// on (run on the CPU by the tests, and in PF_SELFCHECK builds before upload).
//
//   sorted terminals   terminal t = 2l (h = from[l] end) or 2l+1 (k = to[l]
//                      end), ordered by (owner bus, other bus, branch): the
//                      terminal-to-bus permutation of the reduction (Eq. 7);
//                      a bus's terminals, and the parallel runs among them,
//                      are contiguous
//   Ybus pattern       row i = {i} U {other bus of i's terminals}, sorted;
//                      parallel branches share an entry; per entry the range
//                      of sorted terminals whose stamps it sums
//   J pattern          closed form of Alg. 2 (see include/pfgrid.h)
//   element-wise       windows of consecutive buses for one CTA each, with
//                      their ghost buses (other ends outside the window)
#include <algorithm>
#include <cstdint>
#include <limits>

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
    H.tnbr.assign(T, make_int2(0, 0));
    H.town.assign(T, 0);
    H.tmir.assign(T, 0);
    for (int p = 0; p < T; ++p) {
        const int t = H.tsort[p];
        H.tpos[t] = p;
        H.tnbr[p] = make_int2(H.other(t), H.tkpos[t] | (H.taccum[t] ? EW_ACCUM : 0));
        H.town[p] = H.owner(t);
    }
    for (int p = 0; p < T; ++p) H.tmir[p] = H.tpos[H.tsort[p] ^ 1];
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

namespace {

// FP64 instructions of a window's work in the element-wise kernel: per
// terminal (evaluation and its share of the bus sums), per own bus (phasor,
// diagonal entries, S), per ghost bus (phasor)
constexpr long long kCostTerminal = 12, kCostBus = 33, kCostGhost = 17;

// Greedy cut into windows of consecutive buses with at most tb buses, tcap
// terminals and `cap` cost each (a single bus always forms a window); mark[]
// (size nb) is scratch.  A window's cost grows with every bus added, so a
// larger cap never gives more windows.
void cut_windows(const HostTopo &H, int tb, int tcap, long long cap, std::vector<int> &wb, std::vector<int> &mark)
{
    const int nb = H.nb;
    wb.assign(1, 0);
    std::fill(mark.begin(), mark.end(), -1);
    int b = 0, w = 0;
    while (b < nb) {
        const int b0 = b;
        int nt = 0;
        long long cost = 0;
        while (b < nb && b - b0 < tb) {
            const int p0 = H.tp[b], p1 = H.tp[b + 1], th = p1 - p0;
            long long add = kCostBus + kCostTerminal * th - (mark[b] == w ? kCostGhost : 0);
            for (int p = p0; p < p1; ++p) {
                const int q = H.tnbr[p].x;
                if ((q >= b0 && q < b) || mark[q] == w || (p > p0 && H.tnbr[p - 1].x == q)) continue;
                add += kCostGhost;
            }
            if (b > b0 && (nt + th > tcap || cost + add > cap)) break;
            for (int p = p0; p < p1; ++p) {
                const int q = H.tnbr[p].x;
                if (q < b0 || q > b) mark[q] = w;
            }
            nt += th;
            cost += add;
            ++b;
        }
        wb.push_back(b);
        ++w;
    }
}

}  // namespace

pf_status host_ew(const HostTopo &H, int tb, HostEw &E, int tfac, int target_nwin)
{
    if (tb != 128 && tb != 256)
        return set_error(PF_EINVAL, "ew_window (threads per element-wise CTA) must be 128 or 256 (got %d)", tb);
    if (tfac < 1 || tfac > 4) return set_error(PF_EINVAL, "terminals per thread must be 1 .. 4 (got %d)", tfac);
    const int nb = H.nb;
    E = HostEw{};
    E.tb = tb;
    E.tfac = tfac;
    std::vector<int> mark(nb);
    cut_windows(H, tb, tfac * tb, std::numeric_limits<long long>::max(), E.win_bus, mark);
    if (target_nwin > 0 && (int)E.win_bus.size() - 1 < target_nwin) {
        // balance: the smallest cost cap that still gives at most target_nwin windows
        long long lo = 1, hi = 0;
        for (int b = 0; b < nb; ++b) hi += kCostBus + (kCostTerminal + kCostGhost) * (H.tp[b + 1] - H.tp[b]);
        std::vector<int> wb;
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            cut_windows(H, tb, tfac * tb, mid, wb, mark);
            if ((int)wb.size() - 1 <= target_nwin)
                hi = mid;
            else
                lo = mid + 1;
        }
        cut_windows(H, tb, tfac * tb, lo, wb, mark);
        if ((int)wb.size() - 1 <= target_nwin) E.win_bus.swap(wb);
    }
    E.nwin = (int)E.win_bus.size() - 1;
    // per window: sizes, ghost buses, the window-local slot of every terminal's other bus
    E.hptr.assign(E.nwin + 1, 0);
    E.hbus.clear();
    E.tloc.assign(H.tp[nb], make_int2(0, 0));
    std::vector<int> ghosts;
    for (int w = 0; w < E.nwin; ++w) {
        const int b0 = E.win_bus[w], b1 = E.win_bus[w + 1], nbus = b1 - b0;
        const int nt = H.tp[b1] - H.tp[b0];
        E.max_nt = std::max(E.max_nt, nt);
        E.max_nbus = std::max(E.max_nbus, nbus);
        E.max_L = std::max(E.max_L, 2 * (H.rp[b1] - H.rp[b0]));
        ghosts.clear();
        for (int p = H.tp[b0]; p < H.tp[b1]; ++p) {
            const int q = H.tnbr[p].x;
            if (q < b0 || q >= b1) ghosts.push_back(q);
        }
        std::sort(ghosts.begin(), ghosts.end());
        ghosts.erase(std::unique(ghosts.begin(), ghosts.end()), ghosts.end());
        for (int p = H.tp[b0]; p < H.tp[b1]; ++p) {
            const int q = H.tnbr[p].x;
            const int slot = (q >= b0 && q < b1)
                                 ? q - b0
                                 : nbus + (int)(std::lower_bound(ghosts.begin(), ghosts.end(), q) - ghosts.begin());
            E.tloc[p] = make_int2(slot, H.tnbr[p].y);
        }
        E.hbus.insert(E.hbus.end(), ghosts.begin(), ghosts.end());
        E.hptr[w + 1] = (int)E.hbus.size();
        E.max_nh = std::max(E.max_nh, (int)ghosts.size());
        E.max_nph = std::max(E.max_nph, nbus + (int)ghosts.size());
    }
    // fixed-stride per-window records: the descriptor and the bus of every phasor slot
    // (padding slots repeat the window's first bus)
    E.desc.assign(2 * (size_t)E.nwin, make_int4(0, 0, 0, 0));
    E.slotbus.assign((size_t)E.nwin * E.max_nph, 0);
    for (int w = 0; w < E.nwin; ++w) {
        const int b0 = E.win_bus[w], b1 = E.win_bus[w + 1], nbus = b1 - b0;
        const int h0 = E.hptr[w], nph = nbus + E.hptr[w + 1] - h0;
        E.desc[2 * w] = make_int4(b0, nbus, H.tp[b0], H.tp[b1] - H.tp[b0]);
        E.desc[2 * w + 1] = make_int4(H.rp[b0], 2 * (H.rp[b1] - H.rp[b0]), nph, 0);
        int *sb = E.slotbus.data() + (size_t)w * E.max_nph;
        for (int j = 0; j < E.max_nph; ++j) sb[j] = j < nbus ? b0 + j : (j < nph ? E.hbus[h0 + j - nbus] : b0);
    }
    E.bmeta.assign(nb, make_int4(0, 0, 0, 0));
    for (int w = 0; w < E.nwin; ++w)
        for (int o = E.win_bus[w]; o < E.win_bus[w + 1]; ++o)
            E.bmeta[o] = make_int4(2 * (H.rp[o] - H.rp[E.win_bus[w]]), H.rp[o + 1] - H.rp[o], H.kd[o],
                                   H.tp[o] - H.tp[E.win_bus[w]]);
    E.rorder.resize(nb);
    for (int w = 0; w < E.nwin; ++w) {
        const int b0 = E.win_bus[w], b1 = E.win_bus[w + 1];
        int *ord = E.rorder.data() + b0;
        for (int j = 0; j < b1 - b0; ++j) ord[j] = j;
        std::stable_sort(ord, ord + (b1 - b0), [&](int x, int y) {
            return H.tp[b0 + x + 1] - H.tp[b0 + x] > H.tp[b0 + y + 1] - H.tp[b0 + y];
        });
    }
    return PF_OK;
}

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
    CHECK((int)H.tp.size() == nb + 1 && H.tp[0] == 0 && H.tp[nb] == T, "terminal offsets");
    for (int i = 0; i < nb; ++i) {
        CHECK(H.rp[i + 1] > H.rp[i], "row %d empty (diagonal missing)", i);
        CHECK(H.tp[i + 1] >= H.tp[i], "terminal offsets not monotone at %d", i);
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
    for (int p = 0; p < T; ++p) {
        const int o = H.town[p], q = H.tnbr[p].x, kp = H.tnbr[p].y & EW_KMASK;
        CHECK(o >= 0 && o < nb && p >= H.tp[o] && p < H.tp[o + 1], "owner of sorted terminal %d", p);
        CHECK(q >= 0 && q < nb && q != o, "other bus of sorted terminal %d", p);
        CHECK(kp >= 0 && kp < H.rp[o + 1] - H.rp[o] && kp != H.kd[o], "slot of sorted terminal %d", p);
        const bool acc = (H.tnbr[p].y & EW_ACCUM) != 0;
        CHECK(acc == (p > H.tp[o] && H.tnbr[p - 1].x == q), "parallel-run flag of sorted terminal %d", p);
        const int m = H.tmir[p];
        CHECK(m >= 0 && m < T && H.town[m] == q && H.tnbr[m].x == o && H.tmir[m] == p, "mirror of terminal %d", p);
    }
    // element-wise windows: every access of k_jac_ew / k_inj_ew stays in bounds
    CHECK(E.nwin == (int)E.win_bus.size() - 1 && E.win_bus[0] == 0 && E.win_bus[E.nwin] == nb, "window cover");
    for (int w = 0; w < E.nwin; ++w) {
        const int b0 = E.win_bus[w], b1 = E.win_bus[w + 1];
        const int nbus = b1 - b0, nt = H.tp[b1] - H.tp[b0];
        const int L = 2 * (H.rp[b1] - H.rp[b0]);
        CHECK(nbus >= 1 && nbus <= E.tb && nbus <= E.max_nbus, "window %d bus count %d", w, nbus);
        CHECK(nt <= E.max_nt && (nt <= E.tfac * E.tb || nbus == 1), "window %d terminal count %d", w, nt);
        CHECK(L >= 2 && L <= E.max_L, "window %d slice length", w);
        // bulk-store constraints: the J slices start on 16 bytes and are 16-byte multiples
        CHECK((2LL * H.rp[b0]) % 2 == 0 && (8LL * L) % 16 == 0, "window %d J slice alignment", w);
        for (int o = b0; o < b1; ++o) {
            const int lrow = 2 * (H.rp[o] - H.rp[b0]), d = H.rp[o + 1] - H.rp[o];
            CHECK(E.bmeta[o].x == lrow && E.bmeta[o].y == d && E.bmeta[o].z == H.kd[o] &&
                      E.bmeta[o].w == H.tp[o] - H.tp[b0], "bus %d window metadata", o);
            const int j = o - b0, x = E.rorder[o];
            CHECK(x >= 0 && x < b1 - b0, "window %d reduction order entry %d", w, j);
            if (j > 0) {
                const int y = E.rorder[o - 1];
                CHECK(H.tp[b0 + y + 1] - H.tp[b0 + y] >= H.tp[b0 + x + 1] - H.tp[b0 + x],
                      "window %d reduction order not by decreasing terminal count", w);
            }
            CHECK(lrow >= 0 && lrow + 2 * d <= L, "bus %d row slice outside the window slice", o);
            CHECK(lrow + H.kd[o] + d < L, "bus %d diagonal staging index", o);
            for (int p = H.tp[o]; p < H.tp[o + 1]; ++p) {
                const int kp = H.tnbr[p].y & EW_KMASK;
                CHECK(lrow + kp + d < L, "terminal %d staging index", p);
                CHECK(p - H.tp[b0] >= 0 && p - H.tp[b0] < E.max_nt, "terminal %d local index", p);
            }
        }
        {
            std::vector<char> seen(nbus, 0);
            for (int o = b0; o < b1; ++o) seen[E.rorder[o]]++;
            for (int j = 0; j < nbus; ++j) CHECK(seen[j] == 1, "window %d reduction order is not a permutation", w);
        }
    }
    // ghost buses: sorted, outside the window, and every terminal's slot
    // names its other bus
    CHECK((int)E.hptr.size() == E.nwin + 1 && E.hptr[0] == 0 && E.hptr[E.nwin] == (int)E.hbus.size(),
          "ghost-bus offsets");
    CHECK((int)E.tloc.size() == T, "terminal slots");
    CHECK(E.desc.size() == 2 * (size_t)E.nwin && E.slotbus.size() == (size_t)E.nwin * E.max_nph &&
              (int)E.bmeta.size() == nb, "window records");
    for (int w = 0; w < E.nwin; ++w) {
        const int b0 = E.win_bus[w], b1 = E.win_bus[w + 1], nbus = b1 - b0;
        const int h0 = E.hptr[w], nh = E.hptr[w + 1] - h0;
        CHECK(nh >= 0 && nh <= E.max_nh, "window %d ghost count %d", w, nh);
        for (int j = 0; j < nh; ++j) {
            const int q = E.hbus[h0 + j];
            CHECK(q >= 0 && q < nb && (q < b0 || q >= b1), "window %d ghost %d", w, j);
            if (j > 0) CHECK(q > E.hbus[h0 + j - 1], "window %d ghosts not strictly sorted", w);
        }
        const int4 d0 = E.desc[2 * w], d1 = E.desc[2 * w + 1];
        CHECK(d0.x == b0 && d0.y == nbus && d0.z == H.tp[b0] && d0.w == H.tp[b1] - H.tp[b0], "window %d descriptor", w);
        CHECK(d1.x == H.rp[b0] && d1.y == 2 * (H.rp[b1] - H.rp[b0]) && d1.z == nbus + nh && nbus + nh <= E.max_nph,
              "window %d descriptor (rows, slots)", w);
        for (int j = 0; j < E.max_nph; ++j) {
            const int q = E.slotbus[(size_t)w * E.max_nph + j];
            CHECK(q >= 0 && q < nb, "window %d slot %d bus", w, j);
            if (j < nbus) CHECK(q == b0 + j, "window %d own slot %d", w, j);
            else if (j < nbus + nh) CHECK(q == E.hbus[h0 + j - nbus], "window %d ghost slot %d", w, j);
        }
        for (int p = H.tp[b0]; p < H.tp[b1]; ++p) {
            const int slot = E.tloc[p].x, q = H.tnbr[p].x;
            CHECK(E.tloc[p].y == H.tnbr[p].y, "terminal %d slot flags", p);
            CHECK(slot >= 0 && slot < nbus + nh, "terminal %d phasor slot %d", p, slot);
            CHECK(slot < nbus ? b0 + slot == q : E.hbus[h0 + slot - nbus] == q, "terminal %d slot bus", p);
        }
    }
    const EwSmem plan = ew_smem_plan(E.max_nbus, E.max_nt, E.max_L, true, E.max_nph);
    CHECK(plan.total <= kMaxSmem, "a window needs %u bytes of shared memory", plan.total);
    CHECK(plan.yd % 16 == 0 && plan.kg % 16 == 0 && plan.jst % 16 == 0 && plan.pq % 16 == 0 && plan.ph % 16 == 0,
          "shared-memory plan alignment");
    return PF_OK;
}

// Per window, the branches whose from-terminal lies in it, in sorted-terminal
// order: {window-local terminal index, branch}; window w's at
// brl[w * max_nbr ...] (padding {0, 0}), their number in nbr[w].  Every
// branch appears exactly once over the windows.
pf_status host_window_branches(const HostTopo &H, const HostEw &E, std::vector<int2> &brl, std::vector<int> &nbr,
                               int &max_nbr)
{
    nbr.assign(E.nwin, 0);
    max_nbr = 0;
    for (int w = 0; w < E.nwin; ++w) {
        const int t0 = E.desc[2 * w].z, nt = E.desc[2 * w].w;
        int c = 0;
        for (int p = t0; p < t0 + nt; ++p) c += !(H.tsort[p] & 1);
        nbr[w] = c;
        max_nbr = std::max(max_nbr, c);
    }
    brl.assign((size_t)E.nwin * std::max(max_nbr, 1), make_int2(0, 0));
    std::vector<char> seen(H.nl, 0);
    for (int w = 0; w < E.nwin; ++w) {
        const int t0 = E.desc[2 * w].z, nt = E.desc[2 * w].w;
        int j = 0;
        for (int p = t0; p < t0 + nt; ++p) {
            const int t = H.tsort[p];
            if (t & 1) continue;
            brl[(size_t)w * std::max(max_nbr, 1) + j++] = make_int2(p - t0, t >> 1);
            if (seen[t >> 1]++) return set_error(PF_EINVAL, "window branch lists: branch %d listed twice", t >> 1);
        }
    }
    for (int l = 0; l < H.nl; ++l)
        if (!seen[l]) return set_error(PF_EINVAL, "window branch lists: branch %d in no window", l);
    return PF_OK;
}

}  // namespace pf
