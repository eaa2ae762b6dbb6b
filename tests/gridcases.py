"""Small hand-built grids and helpers shared by the tests (inputs only)."""
import numpy as np

from paper_2302_10736_gb300 import synth


def make_grid(nb, branches, shunts=None):
    """branches: list of (h, k, g, b, bsh, tap, shift); shunts: {bus: (gs, bs)}."""
    nl = len(branches)
    gr = dict(nb=nb, nl=nl,
              f=np.array([br[0] for br in branches], np.int32).reshape(nl),
              t=np.array([br[1] for br in branches], np.int32).reshape(nl),
              g=np.array([br[2] for br in branches], float).reshape(nl),
              b=np.array([br[3] for br in branches], float).reshape(nl),
              bsh=np.array([br[4] for br in branches], float).reshape(nl),
              tap=np.array([br[5] for br in branches], float).reshape(nl),
              shift=np.array([br[6] for br in branches], float).reshape(nl),
              gs=np.zeros(nb), bs=np.zeros(nb))
    for i, (a, c) in (shunts or {}).items():
        gr["gs"][i], gr["bs"][i] = a, c
    return gr


def series(r, x):
    z = complex(r, x)
    y = 1.0 / z
    return y.real, y.imag


def two_bus_lossless():
    """Line r = 0, x = 0.1 (y_s = -j10), no charging, nominal ratio."""
    return make_grid(2, [(0, 1, 0.0, -10.0, 0.0, 1.0, 0.0)])


def three_bus_plus():
    """3 meshed buses + 1 isolated bus: a charged line, a parallel pair between
    buses 0 and 1, a phase-shifting tap transformer 1->2 (m = 1.05,
    phi = 0.1) and bus shunts (bus 2, and the isolated bus 3)."""
    gA, bA = series(0.01, 0.1)
    gD, bD = series(0.02, 0.15)
    gB, bB = series(0.005, 0.08)
    gC, bC = series(0.015, 0.12)
    return make_grid(4, [
        (0, 1, gA, bA, 0.04, 1.0, 0.0),
        (1, 2, gB, bB, 0.02, 1.05, 0.1),
        (2, 0, gC, bC, 0.06, 1.0, 0.0),
        (1, 0, gD, bD, 0.03, 0.97, -0.05),   # parallel to the first, reversed
    ], shunts={2: (0.01, 0.05), 3: (0.02, -0.03)})


def random_grid(nb, nl, seed, shift_max=0.0, tx_frac=0.2):
    return synth.grid(nb, nl, seed, tx_frac=tx_frac, shift_max=shift_max)


def random_state(nb, seed, nscen=1, stream=0, sigma=0.2):
    vm, va = synth.voltages(nb, nscen, seed, stream, 0.95, 1.05, sigma)
    return (vm[0], va[0]) if nscen == 1 else (vm, va)


def circuit_currents(gr, vm, va):
    """Bus current injections from the physical branch model, independent of
    any admittance-matrix stamping: an ideal transformer m e^{j phi} : 1 at
    the h end (power conserving), then a pi section with series y_s and half
    of the charging at each end, plus the bus shunts; Kirchhoff's current law
    sums the terminal currents at each bus."""
    V = vm * np.exp(1j * va)
    Ibus = (gr["gs"] + 1j * gr["bs"]) * V
    for l in range(gr["nl"]):
        h, k = gr["f"][l], gr["t"][l]
        ys = gr["g"][l] + 1j * gr["b"][l]
        ych = 1j * gr["bsh"][l] / 2.0
        a = gr["tap"][l] * np.exp(1j * gr["shift"][l])
        Vh_line = V[h] / a                       # voltage on the line side of the transformer
        I_h_line = ys * (Vh_line - V[k]) + ych * Vh_line
        I_h = I_h_line / np.conj(a)              # V_h conj(I_h) = V_h' conj(I_h')
        I_k = ys * (V[k] - Vh_line) + ych * V[k]
        Ibus[h] += I_h
        Ibus[k] += I_k
    return V, Ibus


def blocks(J, jci, nb, nnz):
    """Split canonical J values into (J11, J12, J21, J22) value arrays."""
    P, Q = J[:2 * nnz], J[2 * nnz:]
    th = jci[:2 * nnz] < nb
    return P[th], P[~th], Q[th], Q[~th]


def relerr(x, ref):
    x, ref = np.asarray(x), np.asarray(ref)
    if ref.size == 0:
        return 0.0
    den = np.max(np.abs(ref))
    num = np.max(np.abs(x - ref))
    return float(num / den) if den > 0 else float(num)


def hub_grid(nspokes, seed, nring=600):
    """A ring of `nring` buses plus one hub bus joined to `nspokes` ring buses
    (some twice: parallel spokes): a window holding the hub alone has more
    terminals, and more ghost buses, than a CTA has threads."""
    rng = np.random.default_rng(seed)
    nb = nring + 1
    hub = nring // 2
    br = []
    for i in range(nring + 1):
        if i == hub:
            continue
        j = i + 1 if i + 1 != hub else i + 2
        if j <= nring:
            g, b = series(rng.uniform(0.001, 0.05), rng.uniform(0.01, 0.3))
            br.append((i, j, g, b, rng.uniform(0, 0.1), 1.0, 0.0))
    targets = rng.choice([i for i in range(nb) if i != hub], size=nspokes, replace=False)
    for n, q in enumerate(targets):
        g, b = series(rng.uniform(0.001, 0.05), rng.uniform(0.01, 0.3))
        tap = rng.uniform(0.9, 1.1) if n % 5 == 0 else 1.0
        e = (hub, int(q)) if n % 2 else (int(q), hub)
        br.append(e + (g, b, rng.uniform(0, 0.1), tap, rng.uniform(-0.1, 0.1) if n % 7 == 0 else 0.0))
        if n % 50 == 0:
            br.append(e + (0.5 * g, 0.5 * b, 0.0, tap, 0.0))
    return make_grid(nb, br, shunts={hub: (0.02, -0.01), 3: (0.01, 0.04)})


def superset_pattern(Y, rng, extra):
    """The CSC form of the Ybus-block pattern plus `extra` random coordinates
    and one coupled bus pair (a TCSC-like device: all four blocks), rows in a
    shuffled order within every column."""
    import oracle
    jrp, jci = oracle.jac_pattern(Y)
    n2 = 2 * Y.nb
    coords = {(R, int(jci[p])) for R in range(n2) for p in range(jrp[R], jrp[R + 1])}
    a, c = 0, Y.nb - 1
    for x in (a, c, Y.nb + a, Y.nb + c):
        for y in (a, c, Y.nb + a, Y.nb + c):
            coords.add((x, y))
    extra = min(extra, n2 * n2 - len(coords))
    while len(coords) < len(jci) + extra:
        coords.add((int(rng.integers(n2)), int(rng.integers(n2))))
    cols = [[] for _ in range(n2)]
    for R, C in coords:
        cols[C].append(R)
    colptr = np.zeros(n2 + 1, np.int32)
    rowidx = []
    for C in range(n2):
        rows = cols[C]
        rng.shuffle(rows)
        rowidx += rows
        colptr[C + 1] = len(rowidx)
    return colptr, np.array(rowidx, np.int32)
