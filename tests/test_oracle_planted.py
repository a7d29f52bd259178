"""Planted mistakes in the oracle, on the CPU: each test copies one oracle
module with a plausible error written into its source (a dropped term, a
wrong sign, coefficient or index, a transposed spacing) and checks that a pin
of the kind ``test_oracle_pins.py`` uses rejects the copy, while the
unaltered module passes the same check.  This is evidence that the pins
constrain the oracle and do not merely agree with it."""

import os
import sys
import types

import numpy as np
import pytest

import oracle
from oracle import coupled, dst, stencils
from paper_2609_16478_b300 import inputs

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))
_COUNT = 0


def _copy(name, replacements=(), **overrides):
    """oracle.<name> re-executed from its source with `replacements` (each
    text must occur exactly once) and module names overridden."""
    path = os.path.join(ORACLE_DIR, name + ".py")
    src = open(path).read()
    for old, new in replacements:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    global _COUNT
    _COUNT += 1
    mod = types.ModuleType("oracle._planted_%s_%d" % (name, _COUNT))
    mod.__package__ = "oracle"
    mod.__file__ = path
    sys.modules[mod.__name__] = mod  # dataclasses look their module up there
    exec(compile(src, path, "exec"), mod.__dict__)
    for k, v in overrides.items():
        setattr(mod, k, v)
    return mod


def _coupled_with(stencil_mod):
    return _copy("coupled", laplacian=stencil_mod.laplacian, weighting=stencil_mod.weighting,
                 one_sided_weights=stencil_mod.one_sided_weights)


def _poly_error(cmod, N=(16, 24)):
    """A degree-4 solution with nonzero data of every kind on an anisotropic
    grid: the scheme reproduces it to rounding (P1, P2, R4-R7)."""
    d = inputs.sample(inputs.config_problem("poly2d"), list(N))
    sol = cmod.solve_direct(cmod.assemble(d), d)
    return float(np.max(np.abs(sol.U - d["u_exact"])))


def _exactness_3d(smod):
    """L_h p = M(Lap p) at one point for a degree-5 polynomial, anisotropic h (P1, 3D)."""
    h = (0.11, 0.07, 0.13)
    x0 = np.array([0.3, -0.2, 0.5])

    def p(x, y, z):
        return x ** 4 * y - 2 * x * y ** 2 * z ** 2 + 3 * z ** 5 - y ** 3 + x * z

    def lap(x, y, z):
        return 12 * x ** 2 * y + (-4 * x * z ** 2 - 6 * y) + (-4 * x * y ** 2 + 60 * z ** 3)

    def at(off):
        return x0 + np.array(off) * np.array(h)

    lhs = sum(c * p(*at(o)) for o, c in smod.laplacian(h).items())
    rhs = sum(c * lap(*at(o)) for o, c in smod.weighting(3).items())
    return abs(lhs - rhs) / max(abs(rhs), 1.0)


def test_controls_pass():
    assert _poly_error(coupled) < 1e-11
    assert _exactness_3d(stencils) < 1e-12


PLANTED_STENCILS = {
    "printed 1/2 prefactor (2D)": [("c[(dx, dy)] = v / 12.0", "c[(dx, dy)] = v / 2.0")],
    "one-sided U3 weight": [("Fraction(2, 9))", "Fraction(2, 7))")],
    "one-sided g_N weight": [("ONE_SIDED_GN = Fraction(11, 3)", "ONE_SIDED_GN = Fraction(11, 4)")],
    "weighting centre": [("c[zero] = (8.0 if d == 2 else 6.0) / 12.0", "c[zero] = (9.0 if d == 2 else 6.0) / 12.0")],
    "2D edge weights of the two axes swapped": [("v = 10 * inv[0] - 2 * inv[1]", "v = 10 * inv[1] - 2 * inv[0]")],
}


@pytest.mark.parametrize("what", sorted(PLANTED_STENCILS))
def test_planted_stencil_mistake_is_caught(what):
    smod = _copy("stencils", PLANTED_STENCILS[what])
    assert _poly_error(_coupled_with(smod)) > 1e-6, what


PLANTED_ASSEMBLY = {
    "boundary V dropped from M(V/alpha)": [("        add(ru[face], 2 * n + qf[face], -c / alpha[jf[face]])\n", "")],
    "edge v data dropped": [("        np.add.at(F, rv[edge], c * vE[jf[edge]])\n", "")],
    "g_D of the u-equation with the wrong sign": [("np.add.at(F, ru[bnd], -c * gD[jf[bnd]])",
                                                   "np.add.at(F, ru[bnd], c * gD[jf[bnd]])")],
    "g_N with the wrong sign": [("F[r] = -al * (w0 * gD[pf] + wg * gN[q] + lapt[q])",
                                 "F[r] = -al * (w0 * gD[pf] - wg * gN[q] + lapt[q])")],
    "tangential Laplacian of g_D dropped": [("F[r] = -al * (w0 * gD[pf] + wg * gN[q] + lapt[q])",
                                             "F[r] = -al * (w0 * gD[pf] + wg * gN[q])")],
    "one-sided weights of U1 and U2 swapped": [("for m, w in ((1, w1), (2, w2), (3, w3)):",
                                                "for m, w in ((1, w2), (2, w1), (3, w3)):")],
    "normal spacing of another axis": [("one_sided_weights(h[a])", "one_sided_weights(h[d - 1 - a])")],
    "M f without its boundary values": [("np.add.at(F, rv, c * f[jf])", "np.add.at(F, rv[inter], c * f[jf[inter]])")],
}


@pytest.mark.parametrize("what", sorted(PLANTED_ASSEMBLY))
def test_planted_assembly_mistake_is_caught(what):
    cmod = _copy("coupled", PLANTED_ASSEMBLY[what])
    assert _poly_error(cmod) > 1e-6, what


@pytest.mark.parametrize("old,new", [("v = 8 * inv[a] - 2 * sum", "v = 8 * inv[a] - 3 * sum"),
                                     ("v = -16 * sum(inv)", "v = -15 * sum(inv)"),
                                     ("continue  # the 19-point", "pass  # the 19-point")])
def test_planted_3d_stencil_mistake_is_caught(old, new):
    smod = _copy("stencils", [(old, new)])
    assert _exactness_3d(smod) > 1e-6


def test_planted_schur_rhs_sign_is_caught():
    """Lemma 1: b = -R(0).  With the sign of the A21 term flipped the identity fails."""
    d = inputs.sample(inputs.config_problem("sincos2d"), [8, 8])
    cmod = _copy("coupled", [("return self.F2 - self.A21 @ self.lu.solve(self.F1)",
                              "return self.F2 + self.A21 @ self.lu.solve(self.F1)")])
    for mod, ok in ((coupled, True), (cmod, False)):
        B = mod.Blocks(mod.assemble(d))
        b, R0 = B.schur_rhs(), B.residual(np.zeros(B.sys.ng))
        assert np.allclose(b, -R0, rtol=1e-12, atol=1e-12 * np.max(np.abs(R0))) == ok


def test_planted_dst_normalisation_is_caught():
    """P3: the DST-I against scipy's (which carries a factor 2)."""
    import scipy.fft
    x = np.random.default_rng(2).normal(size=(3, 15))
    bad = _copy("dst", [("np.outer(j, j) / (n + 1)", "np.outer(j, j) / n")])
    assert np.allclose(2 * dst.dst1(x), scipy.fft.dst(x, type=1, axis=-1), rtol=1e-13, atol=1e-12)
    assert not np.allclose(2 * bad.dst1(x), scipy.fft.dst(x, type=1, axis=-1), rtol=1e-3)


def _tri_error(tmod, N=(16, 8)):
    """A degree-5 triharmonic solution with nonzero data of every kind, two
    clamped faces, on an anisotropic grid: reproduced to rounding."""
    d = inputs.sample_triharmonic(inputs.triharmonic_problem("tripoly2d"), list(N))
    sol = tmod.solve_direct(tmod.assemble(d), d)
    return float(np.max(np.abs(sol.U - d["u_exact"])) / np.max(np.abs(d["u_exact"])))


PLANTED_TRIHARMONIC = {
    "u_s with the outward sign": [("ws * (-gN[q])", "ws * gN[q]")],
    "u_ss term dropped": [(" + wss * gNN[q]", "")],
    "tangential part of Lap^2 u dropped": [(" + wss * gNN[q] + lw[q])", " + wss * gNN[q])")],
    "one-sided weights scaled by h^-3": [("wU = [float(cm) / ha ** 4 for cm in cw]", "wU = [float(cm) / ha ** 3 for cm in cw]")],
    "face V data dropped from M V": [("        np.add.at(F, ru[face], c * vb[jf[face]])\n", "")],
    "U_0 weight without c_1": [("c0 = -sum(c14)", "c0 = -sum(c14[1:])")],
    "edge and corner W data with the wrong sign": [("np.add.at(F, rw[edge], -c * wb[jf[edge]])",
                                                    "np.add.at(F, rw[edge], c * wb[jf[edge]])")],
}


def test_triharmonic_control_passes():
    from oracle import triharmonic
    assert _tri_error(triharmonic) < 1e-11


@pytest.mark.parametrize("what", sorted(PLANTED_TRIHARMONIC))
def test_planted_triharmonic_mistake_is_caught(what):
    assert _tri_error(_copy("triharmonic", PLANTED_TRIHARMONIC[what])) > 1e-6, what


def _residual_of_solution(rmod, name="sincos2d", N=(16, 24)):
    """The slicing residual of the assembled system's direct solution (which
    the pins above fix): zero to rounding, relative to each row's terms."""
    d = inputs.sample(inputs.config_problem(name), list(N))
    sol = coupled.solve_direct(coupled.assemble(d), d)
    ru, rv, rq = rmod.coupled_residual(sol.U, sol.V, d)
    h2 = min((d["hi"][a] - d["lo"][a]) / d["N"][a] for a in range(2)) ** 2
    scale = max(np.max(np.abs(sol.U)) / h2, np.max(np.abs(sol.V)) / h2, np.max(np.abs(d["f"])))
    return max(np.max(np.abs(ru)), np.max(np.abs(rv)), np.max(np.abs(rq))) / scale


PLANTED_RESIDUAL = {
    "M f with the wrong sign": [("r_v = -apply_stencil(V, L) - apply_stencil(f, Mw)",
                                 "r_v = -apply_stencil(V, L) + apply_stencil(f, Mw)")],
    "U_3 read from layer 2": [("w3 * layer(U, a, side, 3)", "w3 * layer(U, a, side, 2)")],
    "tangential Laplacian of g_D dropped": [("(dnn + lapt[off:off + n])", "(dnn)")],
    "V / alpha as V": [("apply_stencil(V / alpha, Mw)", "apply_stencil(V, Mw)")],
    "face offset not advanced": [("            off += n\n", "")],
}


def test_residual_control_passes():
    from oracle import residual
    assert _residual_of_solution(residual) < 1e-12


@pytest.mark.parametrize("what", sorted(PLANTED_RESIDUAL))
def test_planted_residual_mistake_is_caught(what):
    assert _residual_of_solution(_copy("residual", PLANTED_RESIDUAL[what])) > 1e-8, what
