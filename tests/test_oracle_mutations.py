"""Planted mistakes in the oracle must be caught by its pins.

Each case copies ``oracle/wilson_oracle.c``, plants one plausible mistake (a
dropped term, a wrong sign, a transposed link, a wrong neighbour, a wrong
conjugation ...), compiles the copy with gcc into a temporary directory and
runs the pins of ``test_oracle_pins.py`` against it. At least one pin has to
fail for every planted mistake; the unmodified oracle passes them all (that is
``test_oracle_pins.py`` itself). Everything runs on the CPU.
"""

import subprocess

import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = {
    "forward projector sign": ("projector(mu, -sign, Pf); /* 1 - gamma_mu for sign = +1 */",
                               "projector(mu, +sign, Pf); /* 1 - gamma_mu for sign = +1 */"),
    "backward link not conjugated": (
        "apply_block(Pb, U + 9 * (mu * V + yb), 1, 0, in + 12 * (yb / 2), acc);",
        "apply_block(Pb, U + 9 * (mu * V + yb), 0, 0, in + 12 * (yb / 2), acc);"),
    "backward link taken at x": (
        "apply_block(Pb, U + 9 * (mu * V + yb), 1, 0, in + 12 * (yb / 2), acc);",
        "apply_block(Pb, U + 9 * (mu * V + x), 1, 0, in + 12 * (yb / 2), acc);"),
    "link transposed": ("W[a][b] = wdag ? conj(U[3 * b + a]) : U[3 * a + b];",
                        "W[a][b] = wdag ? conj(U[3 * a + b]) : U[3 * b + a];"),
    "backward neighbour in the forward direction": (
        "        long yb = neighbour(L, c, mu, -1);\n        /* forward",
        "        long yb = neighbour(L, c, mu, +1);\n        /* forward"),
    "kappa not squared": ("out_e[k] = in_e[k] - kappa * kappa * out_e[k];",
                          "out_e[k] = in_e[k] - kappa * out_e[k];"),
    "gamma_y sign": ("{{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},",
                     "{{0, 0, 0, 1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},"),
    "adjoint with the wrong projector": (
        "apply_block(Pf, U + 9 * (mu * V + xm), 0, 1, in + 12 * (xm / 2), acc);",
        "apply_block(Pb, U + 9 * (mu * V + xm), 0, 1, in + 12 * (xm / 2), acc);"),
    "outer product without conjugation": ("s += p[3 * j + a] * conj(q[3 * j + b]);",
                                          "s += p[3 * j + a] * q[3 * j + b];"),
    "force projection sign": ("0.5 * (W[3 * a + b] - conj(W[3 * b + a]))",
                              "0.5 * (W[3 * a + b] + conj(W[3 * b + a]))"),
    "CG beta inverted": ("double beta = rr_new / rr;", "double beta = rr / rr_new;"),
    "sites of the wrong parity": ("        if (parity_of(c) != out_parity) continue;\n        hop_site(",
                                  "        if (parity_of(c) == out_parity) continue;\n        hop_site("),
    "gradient with the wrong projector": ("projector(mu, -1, Pm); /* 1 - gamma_mu */",
                                          "projector(mu, +1, Pm); /* 1 - gamma_mu */"),
    # the site-by-site M_eo that checks the full-size lattices
    "sites: kappa not squared": ("out[12 * n + k] = in[12 * (x / 2) + k] - kappa * kappa * acc[k];",
                                 "out[12 * n + k] = in[12 * (x / 2) + k] - kappa * acc[k];"),
    "sites: adjoint's backward link taken at x": (
        "apply_block(Pf, U + 9 * (mu * V + yb), 0, 1, tb[mu], acc);",
        "apply_block(Pf, U + 9 * (mu * V + x), 0, 1, tb[mu], acc);"),
    "sites: odd site for an even index": ("return parity_of(c) == 0 ? 2 * i : 2 * i + 1;",
                                          "return parity_of(c) == 1 ? 2 * i : 2 * i + 1;"),
}


def _pins(o):
    return [
        ("gamma table", lambda: pins.test_gamma_basis_algebra(o)),
        ("dense 2^4", lambda: pins.test_dense_blocks_and_meo(o, (2, 2, 2, 2), "haar")),
        ("dense 2x4x2x6", lambda: pins.test_dense_blocks_and_meo(o, (2, 4, 2, 6), "smooth")),
        ("adjoint identity", lambda: pins.test_adjoint_identity(o)),
        ("gamma5 hermiticity", lambda: pins.test_gamma5_hermiticity(o)),
        ("gauge covariance", lambda: pins.test_gauge_covariance(o)),
        ("free field", lambda: pins.test_free_field_plane_wave(o, (1, 2, 1, 3))),
        ("link gradient FD", lambda: pins.test_link_grad_finite_differences(o)),
        ("force FD", lambda: pins.test_force_finite_differences(o)),
        ("CG vs dense", lambda: pins.test_cg_against_dense_normal_equations(o)),
        ("M_eo site by site vs full", lambda: pins.test_meo_sites_matches_full(o)),
    ]


def _run_pins():
    caught = []
    for name, fn in _pins(oracle):
        try:
            fn()
        except Exception:  # an assertion, or an error a broken oracle provokes
            caught.append(name)
    return caught


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path, oracle_lib):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation site for {name!r} not found"
    (tmp_path / "mut.c").write_text(src.replace(old, new, 1))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(lib),
                    str(tmp_path / "mut.c"), "-lm"], check=True)
    with oracle.use_library(str(lib)):
        caught = _run_pins()
    assert caught, f"planted mistake {name!r} passed every pin"


def test_unmodified_copy_passes_every_pin(tmp_path, oracle_lib):
    lib = tmp_path / "libsame.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(lib),
                    oracle._SRC, "-lm"], check=True)
    with oracle.use_library(str(lib)):
        assert _run_pins() == []
