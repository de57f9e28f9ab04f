"""Pins of the oracle's limiter (Sec. 2.3) and of the mortar flux's reduction
to the conforming flux (Sec. 2.2), each checked to fail on a mistake planted
in a copy of the oracle.

- FCT assembly: with every factor forced to 0 the limited stage is the
  low-order update bit for bit (Eq. LowOrderScheme_globalIndices); forced to
  1 it is the unlimited high-order residual of Eq. evolutionformula, so the
  antidiffusive volume and mortar fluxes are exactly high minus low order.
- Zalesak density factors (reading R7): a node whose R+ (R-) is below one
  lands exactly on rho_max (rho_min) when its positive (negative)
  antidiffusive fluxes alone are applied at that factor; R = 1 admits them
  all; an interface factor never exceeds the receiving node's R+ nor the
  giving node's R-, and is the largest such value unless the pressure factor
  binds (reading R8, checked by evaluating the pressure of the Gamma-scaled
  update independently).
- Mortar factor (reading R9, with the n_i budget of the remark in Sec. 2.3):
  n_i counted from the mesh, every node of a mortar admissible at l_S, and
  some node inadmissible just above l_S when l_S < 1, on meshes with corner
  nodes shared by two mortars, N = 1..5.
- Local weights of a conforming face (App. A with a 1:1 overlap) are
  delta_ij w_i and the sparse interface flux equals the conforming LLF
  (Eq. mortarfluxforconforminginterface).
"""
import os

import numpy as np
import pytest

import oracle
from conftest import rhs_scale
from paper_2607_06045_b300 import workloads as W

G = 1.4
SRC = os.path.join(os.path.dirname(oracle.__file__), "idp_oracle.c")


# ----------------------------------------------------------------------------
# planted mistakes
# ----------------------------------------------------------------------------

def mutant(tmp_path_factory, name, old, new):
    """Build the oracle with one textual change (old must occur exactly once)."""
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {name}: pattern not unique"
    d = tmp_path_factory.mktemp(f"mut_{name}")
    return oracle.compile_source(src.replace(old, new), str(d / f"lib_{name}.so"))


MUTATIONS = {
    # R7: the k-side factor taken from the wrong sign
    "zalesak_swap_k": ("(Rp[gl] < Rm[gr] ? Rp[gl] : Rm[gr]) : (Rm[gl] < Rp[gr] ? Rm[gl] : Rp[gr]);",
                       "(Rp[gl] < Rp[gr] ? Rp[gl] : Rp[gr]) : (Rm[gl] < Rm[gr] ? Rm[gl] : Rm[gr]);"),
    # R7: the interface factor as the minimum of all four node factors
    "zalesak_min4": ("(Rp[gl] < Rm[gr] ? Rp[gl] : Rm[gr]) : (Rm[gl] < Rp[gr] ? Rm[gl] : Rp[gr]);",
                     "fmin(fmin(Rp[gl], Rm[gl]), fmin(Rp[gr], Rm[gr])) : fmin(fmin(Rp[gl], Rm[gl]), fmin(Rp[gr], Rm[gr]));"),
    # R7: Q+ formed with the lower bound
    "zalesak_q": ("double Qp = m / dt * (rmax[i] - rfv), Qm = m / dt * (rmin[i] - rfv);",
                  "double Qp = m / dt * (rmax[i] - rfv) * 0.5, Qm = m / dt * (rmin[i] - rfv);"),
    # R9: no high-order mortar flux at all
    "mortar_zero": ("        if (g_force_ell >= 0.0) lS = g_force_ell;\n",
                    "        lS = 0.0;\n        if (g_force_ell >= 0.0) lS = g_force_ell;\n"),
    # R9: the budget n_i ignored
    "mortar_n1": ("double mi = mass(c, i), ni = (double)c->mcount[i];",
                  "double mi = mass(c, i), ni = 1.0;"),
    # R9: only the large side's nodes limit the factor
    "mortar_large_only": ("            if (th < lS) lS = th;\n",
                          "            if (th < lS && q < np) lS = th;\n"),
    # FCT assembly: the mortar antidiffusive flux with the wrong sign
    "mortar_h_sign": ("                H[k][v] = -(FL2 - Flo[k][v]);",
                      "                H[k][v] = (FL2 - Flo[k][v]);"),
    # interface flux: the dissipation of a pair term halved
    "pair_dissipation": ("        Fi[v] += 0.5 * (wt * (fi[v] + fj[v]) - aw * lam * (uj[v] - ui[v]));",
                         "        Fi[v] += 0.5 * (wt * (fi[v] + fj[v]) - 0.5 * aw * lam * (uj[v] - ui[v]));"),
    # App. A: the other side's subcells not scaled on a conforming face
    "overlap_scale": ("                double sc = ratio == 1 ? 1.0 : 0.5;",
                      "                double sc = 0.5;"),
}


@pytest.fixture(scope="module")
def mutants(tmp_path_factory):
    return {k: mutant(tmp_path_factory, k, *v) for k, v in MUTATIONS.items()}


# ----------------------------------------------------------------------------
# cases
# ----------------------------------------------------------------------------

def corner_mesh():
    """4 x 4 periodic base grid with one element refined: four mortars, and the
    corner nodes of the four small elements each lie on two of them."""
    return W.box_refined_mesh(4, 4, (0.0, 0.0, 1.0, 1.0), (0.3, 0.3, 0.45, 0.45))


def rough_state(m, N, seed):
    return W.random_state(m, N, seed=seed, rho_range=(0.1, 10.0), p_range=(0.1, 10.0), vmax=2.0)


def disc_state(m, N):
    """A density and pressure disc across the refined element's lower-left
    corner on a smooth background, moving diagonally: its mortars are
    limited to factors strictly between 0 and 1 at N = 2..4."""
    X, Y = W.node_coords(m, N)
    inside = ((X - 0.3) ** 2 + (Y - 0.375) ** 2) < 0.15 ** 2
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) + 2.0 * inside
    return W.conserved(rho, 0.3 + 0 * X, -0.2 + 0 * X, 1.0 + 4.0 * inside, G)


_CASES = None


def cases():
    """(mesh, N, state) triples: the refined square with the disc jump across
    the mortar ring (N = 3), the corner mesh with a disc across its mortars
    (N = 1..5), and the corner mesh on a rough seeded state (N = 3)."""
    global _CASES
    if _CASES is None:
        sq = W.square_mesh()
        cm = corner_mesh()
        _CASES = [(sq, 3, W.disc_wave_state(sq, 3))]
        _CASES += [(cm, N, disc_state(cm, N)) for N in (1, 2, 3, 4, 5)]
        _CASES.append((cm, 3, rough_state(cm, 3, seed=11)))
    return _CASES


N_CASES = 7


def pressure(u):
    return (G - 1) * (u[..., 3] - 0.5 * (u[..., 1] ** 2 + u[..., 2] ** 2) / u[..., 0])


# ----------------------------------------------------------------------------
# pin checks (each returns a list of failures)
# ----------------------------------------------------------------------------

def check_fct_reductions(mesh, N, u):
    o = oracle.Oracle(mesh, N)
    dt = o.dt(u, cfl=0.5)
    mm = o.masses()
    bad = []
    for lim in (1, 2):
        r0 = o.stage_debug(u, 0.0, dt, limiting=lim, force_ell=0.0)
        rfv, _ = o.fv_residual(u)
        if not np.array_equal(r0["res"], rfv):
            bad.append(f"l=0 residual differs from the low-order residual (limiting {lim})")
        if not np.array_equal(r0["ut"], u + dt / mm[None] * rfv):
            bad.append(f"l=0 stage differs from the low-order update (limiting {lim})")
        r1 = o.stage_debug(u, 0.0, dt, limiting=lim, force_ell=1.0)
        rdg = o.dg_residual(u)
        sc = rhs_scale(u, o.dt(u, cfl=1.0))[:, None] * mm.reshape(1, -1)
        err = (np.abs(r1["res"] - rdg).reshape(4, -1) / sc).max()
        if err > 1e-12:
            bad.append(f"l=1 residual differs from the high-order residual by {err:.2e} (limiting {lim})")
    return bad


def check_zalesak(mesh, N, u):
    """R7 landing and maximality; exempt interfaces (R15) are skipped."""
    o = oracle.Oracle(mesh, N)
    dt = o.dt(u, cfl=0.5)
    r = o.stage_debug(u, 0.0, dt, limiting=2)
    node, itf = r["node"], r["iface"]
    mm = o.masses().reshape(-1)
    nn = len(mm)
    rfv, rmin, rmax, Rp, Rm = node[:, 0], node[:, 1], node[:, 2], node[:, 6], node[:, 7]
    gl, gr = itf[:, 0].astype(int), itf[:, 1].astype(int)
    A, ex, lrho = itf[:, 2], itf[:, 3] > 0, itf[:, 4]
    Pp, Pm = np.zeros(nn), np.zeros(nn)
    act = ~ex
    for nodes, G_ in ((gl, -A), (gr, A)):
        np.add.at(Pp, nodes[act], np.maximum(G_[act], 0.0))
        np.add.at(Pm, nodes[act], np.minimum(G_[act], 0.0))
    bad = []
    sc = np.maximum(np.abs(rmax), np.abs(rmin))
    # landing on the bound
    hit_p = rfv + dt / mm * Rp * Pp
    hit_m = rfv + dt / mm * Rm * Pm
    lp, lm = Rp < 1.0, Rm < 1.0
    if np.any(np.abs(hit_p - rmax)[lp] > 1e-14 * sc[lp]):
        bad.append("R+ < 1 does not land on rho_max")
    if np.any(np.abs(hit_m - rmin)[lm] > 1e-14 * sc[lm]):
        bad.append("R- < 1 does not land on rho_min")
    if np.any((hit_p - rmax)[~lp] > 1e-14 * sc[~lp]) or np.any((rmin - hit_m)[~lm] > 1e-14 * sc[~lm]):
        bad.append("R = 1 where the full flux leaves the bounds")
    if lp.sum() + lm.sum() == 0:
        bad.append("no node is density-limited: the case does not exercise R7")
    # interface factor: receiver's R+, giver's R-
    into_r = A > 0               # node gr receives +A
    recv = np.where(into_r, gr, gl)
    give = np.where(into_r, gl, gr)
    cap = np.minimum(Rp[recv], Rm[give])
    nz = act & (A != 0)
    if np.any(lrho[nz] > cap[nz] * (1 + 1e-15)):
        bad.append("interface factor above the receiver's R+ or the giver's R-")
    # maximality: the density factor is not below what both budgets allow
    # (the pressure factor of reading R8 acts afterwards and is pinned by its
    # own brute-force scan)
    if np.any(lrho[nz] < cap[nz] * (1 - 1e-15)):
        bad.append("interface factor below min(R+ receiver, R- giver)")
    lfin = itf[:, 7]
    if np.any(lfin[nz] > lrho[nz]):
        bad.append("final interface factor above the density factor")
    return bad


def mortar_nodes_from_mesh(o, N):
    """Global node indices of each mortar (large face, lower small, upper small),
    formed from the mortar list and the node layout (e, j, i)."""
    np_ = N + 1
    out = []
    for dirn, L, low, s0, s1 in o.mortars():
        def side(e, s):
            if s == 0:   # -x
                return [(e * np_ + j) * np_ + 0 for j in range(np_)]
            if s == 1:   # +x
                return [(e * np_ + j) * np_ + N for j in range(np_)]
            if s == 2:   # -y
                return [(e * np_ + 0) * np_ + i for i in range(np_)]
            return [(e * np_ + N) * np_ + i for i in range(np_)]
        sL = (1 if low else 0) if dirn == 0 else (3 if low else 2)
        sS = sL ^ 1
        out.append(side(L, sL) + side(s0, sS) + side(s1, sS))
    return out


def check_mortar_factor(mesh, N, u, entropy=0):
    o = oracle.Oracle(mesh, N)
    dt = o.dt(u, cfl=0.5)
    r = o.stage_debug(u, 0.0, dt, limiting=2, entropy=entropy)
    node, mort, ell = r["node"], r["mortar"], r["mortar_ell"]
    mm = o.masses().reshape(-1)
    bad = []
    lists = mortar_nodes_from_mesh(o, N)
    count = np.zeros(len(mm), int)
    for lst in lists:
        for g in set(lst):
            count[g] += 1
    if count.max() < 2:
        bad.append("no node lies on two mortars: the case does not exercise the n_i budget")
    n_limited = 0
    for m, lst in enumerate(lists):
        rec = mort[m]
        if not np.array_equal(rec[:, 0].astype(int), np.array(lst)):
            bad.append(f"mortar {m}: node list differs from the mesh's")
            continue
        ni = count[lst]
        if not np.array_equal(rec[:, 14].astype(int), ni):
            bad.append(f"mortar {m}: n_i differs from the count of incident mortars")
        a_expect = ni * dt / mm[lst] * rec[:, 15]
        if np.any(np.abs(rec[:, 7] - a_expect) > 1e-14 * np.abs(a_expect).max() + 1e-300):
            bad.append(f"mortar {m}: density correction not scaled by n_i dt / m_i")
        u0, av = rec[:, 3:7], rec[:, 7:11]
        rlo, rhi, pm = rec[:, 11], rec[:, 12], rec[:, 13]
        rfv = node[lst, 0]
        tol = 1e-14 * np.abs(rfv)

        def feasible(l, slack):
            v = u0 + l * av
            ok_r = (v[:, 0] >= rlo - tol - slack * np.abs(rlo)) & (v[:, 0] <= rhi + tol + slack * np.abs(rhi))
            ok_p = pressure(v) >= pm - 1e-14 * np.abs(pm) - slack * np.abs(pm)
            return ok_r & ok_p
        lS = ell[m]
        if not np.all(feasible(lS, 1e-13)):
            bad.append(f"mortar {m}: a node is inadmissible at l_S = {lS}")
        if lS < 1.0:
            n_limited += 1
            up = min(1.0, lS + max(1e-8 * lS, 1e-10))
            if np.all(feasible(up, 0.0)) and not entropy:
                bad.append(f"mortar {m}: l_S = {lS} is not the largest admissible factor")
    if n_limited == 0:
        bad.append("no mortar is limited: the case does not exercise R9")
    # the final state keeps every bound
    if r["stats"]["viol_rho"] or r["stats"]["viol_p"]:
        bad.append("bound violations after the stage")
    return bad


def check_conforming_reduction(N, seed=0):
    rng = np.random.default_rng(seed)
    np_ = N + 1

    def states(n):
        return np.array([W.conserved(rng.uniform(.3, 3), rng.uniform(-1, 1), rng.uniform(-1, 1),
                                     rng.uniform(.3, 3), G) for _ in range(n)])
    uA, uB = states(np_), states(np_)
    F, wt = oracle.face_sparse(N, 1, uA, uB)
    _, w = oracle.lgl(N)
    bad = []
    off = wt - np.diag(np.diag(wt))
    if np.any(off != 0.0) or np.abs(np.diag(wt) - w).max() > 1e-15:
        bad.append("conforming local weights are not delta_ij w_i")
    llf = np.array([w[i] * oracle.llf(uA[i], uB[i], (1.0, 0.0)) for i in range(np_)])
    if np.abs(F[:np_] - llf).max() > 1e-14 * np.abs(llf).max():
        bad.append("sparse flux of a conforming face differs from the LLF flux")
    if np.abs(F[np_:] + llf).max() > 1e-14 * np.abs(llf).max():
        bad.append("the other side's flux is not the negated LLF flux")
    return bad


# ----------------------------------------------------------------------------
# the pins
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("case", range(N_CASES))
def test_fct_reductions(case):
    m, N, u = cases()[case]
    assert check_fct_reductions(m, N, u) == []


@pytest.mark.parametrize("case", range(N_CASES))
def test_zalesak_landing_and_maximality(case):
    m, N, u = cases()[case]
    assert check_zalesak(m, N, u) == []


@pytest.mark.parametrize("case", range(N_CASES))
def test_mortar_factor_maximal(case):
    m, N, u = cases()[case]
    assert check_mortar_factor(m, N, u) == []


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_conforming_reduction(N):
    assert check_conforming_reduction(N) == []


# ----------------------------------------------------------------------------
# each pin catches its planted mistakes
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name,check", [
    ("zalesak_swap_k", "zalesak"), ("zalesak_min4", "zalesak"), ("zalesak_q", "zalesak"),
    ("mortar_zero", "mortar"), ("mortar_n1", "mortar"), ("mortar_large_only", "mortar"),
    ("mortar_h_sign", "fct"), ("pair_dissipation", "reduction"), ("overlap_scale", "reduction"),
])
def test_pins_catch_planted_mistakes(mutants, name, check):
    fn = {"zalesak": check_zalesak, "mortar": check_mortar_factor, "fct": check_fct_reductions}
    with oracle.using(mutants[name]):
        if check == "reduction":
            failures = sum((check_conforming_reduction(N) for N in (1, 3, 5)), [])
        else:
            failures = sum((fn[check](m, N, u) for m, N, u in cases()), [])
    assert failures, f"mutation {name} passed the {check} pins"
