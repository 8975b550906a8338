"""Planted mistakes in the oracle (CPU only) must each fail at least one pin.

Each mutant is the oracle's C source with one plausible error substituted in
(a dropped term, a wrong sign, index or factor, a transposed operand, or an
alternative reading of the paper that the pins rule out), compiled into a
temporary library.  The fast pins run against it; a mutant that passes every
pin would mean the pins cannot tell that mistake from the method.
"""
import os

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "lbm_oracle.c")

MUTANTS = {
    "w(2)=1/6": ("if (e2 == 2) return 1.0 / 12.0;", "if (e2 == 2) return 1.0 / 6.0;"),
    "force sign": ("Fx[y * nx + x] = -G * psi", "Fx[y * nx + x] = G * psi"),
    "force y uses e_x": ("sy += w_int(a) * pn * ey[a];", "sy += w_int(a) * pn * ex[a];"),
    "stream backwards in x": ("int xd = ((x + ex[a]) % nx + nx) % nx;",
                              "int xd = ((x - ex[a]) % nx + nx) % nx;"),
    "SC shift without tau": ("oracle_feq(rho, ux + tau * Fx / rho, uy + tau * Fy / rho, feq);",
                             "oracle_feq(rho, ux + Fx / rho, uy + Fy / rho, feq);"),
    "EDM du = F/(2 rho)": ("oracle_feq(rho, ux + Fx / rho, uy + Fy / rho, feq2);",
                           "oracle_feq(rho, ux + Fx / (2.0 * rho), uy + Fy / (2.0 * rho), feq2);"),
    "upsilon = c_s^2 (tau - 1/2)": ("double ups = tau - 0.5;", "double ups = (tau - 0.5) / 3.0;"),
    "improved f_eq at u": ("oracle_feq(rho, vx, vy, feq); /* Guo",
                           "oracle_feq(rho, ux, uy, feq); /* Guo"),
    "improved without (1 - 1/2tau)": ("double Fa = (1.0 - 1.0 / (2.0 * tau)) * improved_bracket(",
                                      "double Fa = improved_bracket("),
    "v' with psi not psi^2": ("*vpx = *vx + sigma * Fx / (ups * psi * psi);",
                              "*vpx = *vx + sigma * Fx / (ups * psi);"),
    "f_eq drops c_s^2 u.u": ("(eu * eu - cs2() * uu)", "(eu * eu - uu)"),
    "weight 1/36 -> 1/18": ("1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};",
                            "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 18.0};"),
    "CS numerator sign": ("1.0 + eta + eta * eta - eta * eta * eta",
                          "1.0 + eta + eta * eta + eta * eta * eta"),
    "psi without rho c_s^2": ("(oracle_p_eos(rho, RT, a, b) - rho * cs2())",
                              "(oracle_p_eos(rho, RT, a, b) - rho)"),
    "moment u_y from j_x": ("uy[c] = jy / r;", "uy[c] = jx / r;"),
    "collision u_y from e_x": ("jy += f[a] * ey[a];", "jy += f[a] * ex[a];"),
    "Ladd with v in F_a": ("guo_term(a, 1.0, 1.0, ux, uy, Fx, Fy)",
                           "guo_term(a, 1.0, 1.0, ux + Fx / (2.0 * rho), uy + Fy / (2.0 * rho), Fx, Fy)"),
    "modified EDM with C_e = 1": ("guo_term(a, 1.0, 1.0 / tau, vx, vy, Fx, Fy)",
                                  "guo_term(a, 1.0, 1.0, vx, vy, Fx, Fy)"),
    "Guo term B_e <- C_e": ("return wq[a] * (Be * Fe / cs2()", "return wq[a] * (Ce * Fe / cs2()"),
    "actual velocity u + F/rho": ("vy[c] = uy[c] + Fy[c] / (2.0 * rho[c]);",
                                  "vy[c] = uy[c] + Fy[c] / rho[c];"),
    "MRT without the half-rate factor": ("(1.0 - 0.5 * S[k]) * mf", "mf"),
    "MRT energy rates swapped": ("double S[Q] = {sv, se, seps, sv, sq, sv, sq, sv, sv};",
                                 "double S[Q] = {sv, seps, se, sv, sq, sv, sq, sv, sv};"),
    "MRT energy row 3|c|^2 -> 2|c|^2": ("M[1][a] = -4.0 + 3.0 * c2;", "M[1][a] = -4.0 + 2.0 * c2;"),
    "MRT f_eq moments at u": ("oracle_feq(rho, vx, vy, feq);\n  for (int a = 0; a < Q; ++a) fhat",
                              "oracle_feq(rho, ux, uy, feq);\n  for (int a = 0; a < Q; ++a) fhat"),
    "at-rest velocity +F/(2 rho)": ("ux[c] = -Fx[c] / (2.0 * rho[c]);\n    uy[c] = -Fy[c] / (2.0 * rho[c]);",
                                    "ux[c] = Fx[c] / (2.0 * rho[c]);\n    uy[c] = Fy[c] / (2.0 * rho[c]);"),
    "at-rest velocity -F/rho": ("ux[c] = -Fx[c] / (2.0 * rho[c]);\n    uy[c] = -Fy[c] / (2.0 * rho[c]);",
                                "ux[c] = -Fx[c] / rho[c];\n    uy[c] = -Fy[c] / rho[c];"),
    "mass skips the rest population": ("for (size_t i = 0; i < Q * n; ++i) m += f[i];",
                                       "for (size_t i = n; i < Q * n; ++i) m += f[i];"),
    "EOS attraction sign": ("return rho * RT * num / den - a * rho * rho;",
                            "return rho * RT * num / den + a * rho * rho;"),
    "EOS denominator (1 - eta)^2": ("double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);",
                                    "double den = (1.0 - eta) * (1.0 - eta);"),
    "eta = b rho / 2": ("double eta = b * rho / 4.0;", "double eta = b * rho / 2.0;"),
    "psi without the factor 2": ("double arg = 2.0 * (", "double arg = 1.0 * ("),
    "w(1) = 1/4": ("if (e2 == 1) return 1.0 / 3.0;", "if (e2 == 1) return 1.0 / 4.0;"),
    "stream backwards in y": ("int yd = ((y + ey[a]) % ny + ny) % ny;",
                              "int yd = ((y - ey[a]) % ny + ny) % ny;"),
    "f_eq linear term without 1/c_s^2": ("(1.0 + eu / cs2() +", "(1.0 + eu +"),
    "Guo second-order term halved": ("double Cee = 2.0 * Ce *", "double Cee = Ce *"),
    "modified EDM f_eq at v": ("oracle_feq(rho, ux, uy, feq);\n      for (int a = 0; a < Q; ++a)\n        fout[a] = f[a] - (f[a] - feq[a]) / tau +\n                  guo_term(a, 1.0, 1.0 / tau",
                               "oracle_feq(rho, vx, vy, feq);\n      for (int a = 0; a < Q; ++a)\n        fout[a] = f[a] - (f[a] - feq[a]) / tau +\n                  guo_term(a, 1.0, 1.0 / tau"),
    "improved v = u + F/rho": ("*vx = ux + Fx / (2.0 * rho);", "*vx = ux + Fx / rho;"),
    "SC shift against the force": ("oracle_feq(rho, ux + tau * Fx / rho, uy + tau * Fy / rho, feq);",
                                   "oracle_feq(rho, ux - tau * Fx / rho, uy - tau * Fy / rho, feq);"),
    "SC relaxation 1/tau -> tau": ("for (int a = 0; a < Q; ++a) fout[a] = f[a] - (f[a] - feq[a]) / tau;\n      return 0;\n    }\n    case OR_EDM: {",
                                   "for (int a = 0; a < Q; ++a) fout[a] = f[a] - (f[a] - feq[a]) * tau;\n      return 0;\n    }\n    case OR_EDM: {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name!r} not unique"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib_path = oracle.compile_oracle(str(mutant), str(tmp_path / "libmutant.so"))
    lib = oracle.load(lib_path)
    caught = []
    for pin in P.ALL_FAST_PINS:
        try:
            fails = pin(lib)
        except Exception as e:  # a crash in a pin also exposes the mutant
            fails = [repr(e)]
        if fails:
            caught.append(pin.__name__)
    assert caught, f"mutant {name!r} passed every pin"
