"""The pins catch plausible mistakes: each case plants one mistake in a copy
of the oracle's C source (a dropped term, a wrong sign or factor, a missed
update), builds it into a temporary library, and runs a pin against it,
which must fail.  The real oracle is untouched and restored afterwards.

A planted edit whose text is no longer in the source fails the test, so the
mutations cannot silently go stale.
"""
import os
import shutil
import subprocess

import pytest

import oracle

import test_oracle_assembly as T_asm
import test_oracle_flux as T_flux
import test_oracle_junction as T_junc
import test_oracle_krylov as T_kry
import test_oracle_normal_permeability as T_kn
import test_oracle_precision as T_prec
import test_oracle_schur_amg as T_amg
import test_oracle_smoothers as T_sm
from paper_2206_03203_gb300 import inputs

MUTATIONS = {
    # the matrix-fracture coupling of the matrix rows with twice the interface resistance
    "coupling factor": (
        "row[cnt].t = F / (h / (2.0 * ki) + 1.0 / kappa);",
        "row[cnt].t = F / (h / (2.0 * ki) + 2.0 / kappa);",
        lambda o: T_asm.test_series_fracture_closed_form(o, 3.0, 0.05)),
    # Eq. (7) with the wrong sign of the correction
    "Schur sign": (
        "acc[j] = acc[j] - (Amf->v[p] * Afm->v[q]) / dk[k];",
        "acc[j] = acc[j] + (Amf->v[p] * Afm->v[q]) / dk[k];",
        lambda o: T_amg.test_schur_dense_brute_force(o, lambda: inputs.fixed_2d(n=16))),
    # star-delta with the pairwise denominator
    "star-delta denominator": (
        "row[cnt].t = junction ? (tk * tl) / S : (tk * tl) / (tk + tl);",
        "row[cnt].t = (tk * tl) / (tk + tl);",
        lambda o: T_junc.test_crossing_star_delta_closed_form(o)),
    # the Chebyshev recurrence without the update of rho
    "Chebyshev recurrence": (
        "        rho = rho_new;\n    }\n    free(d);",
        "    }\n    free(d);",
        lambda o: T_sm.test_chebyshev_residual_polynomial(o, 3)),
    # the normal permeability ignored
    "normal permeability dropped": (
        "const double *kn = fc_kn ? fc_kn : fc_kf;",
        "const double *kn = fc_kf;",
        lambda o: T_kn.test_across_a_fracture_only_kn_counts(o, 1e4, 1e-4, 1e-4)),
    # the strength threshold dropped: every coupling strong
    "strength threshold": (
        "double th2 = theta * theta;",
        "double th2 = 0.0 * theta;",
        lambda o: T_amg.test_strength_anisotropic(o)),
    # a wrong sign in the Givens rotation of the Hessenberg column
    "Givens rotation sign": (
        "H[(q + 1) * m + j] = -sn[q] * a + cs[q] * c;",
        "H[(q + 1) * m + j] = sn[q] * a + cs[q] * c;",
        lambda o: T_kry.test_identity_fgmres_is_gmres_finite_termination(o)),
    # the paper's partition: the fracture side of a flux with the wrong sign
    "flux sign": (
        "row[cnt].t = -1.0;",
        "row[cnt].t = 1.0;",
        lambda o: T_flux.test_flux_form_structure(o, "fixed2d-16")),
    # an intersection flux row with half the member's transmissibility
    "intersection flux law": (
        "A->v[pos++] = -1.0 / tl;",
        "A->v[pos++] = -1.0 / (2.0 * tl);",
        lambda o: T_junc.test_intersection_form_structure(o, "fixed2d-16")),
    # smoothed aggregation with the damping 1 instead of 4/3
    "SA damping": (
        "double ci = (4.0 / 3.0) / d1;",
        "double ci = 1.0 / d1;",
        lambda o: T_amg.test_smoothed_prolongator_and_galerkin(o, lambda: T_amg.lap2(12))),
    # bf16 rounding that truncates instead of rounding to nearest even
    "bf16 rounding": (
        "u = (u + 0x7fffu + lsb) & 0xffff0000u;",
        "u = u & 0xffff0000u;",
        lambda o: T_amg.test_lowp_rounding(o)),
    # restriction that drops the last member of each aggregate's sum (r_i of
    # odd i left out)
    "restriction": (
        "if (h->agg[l][i] >= 0) bc[h->agg[l][i]] += r[i];",
        "if (h->agg[l][i] >= 0 && (i & 1) == 0) bc[h->agg[l][i]] += r[i];",
        lambda o: T_amg.test_vcycle_two_grid_error_propagation(o, 0)),
    # bf16 / fp16 row scales rounded down instead of up: 2^floor(log2 max|a_ij|)
    "row scale exponent": (
        "if (fr == 0.5) e -= 1;",
        "e -= 1;",
        lambda o: T_prec.test_row_scaled_storage_rule(o, 17, "rects3d-12")),
    # the restricted right-hand side handed to the coarse level unrounded
    "coarse rhs not rounded": (
        "for (int64_t I = 0; I < nc; I++) bc[I] = rnd(bc[I], pv);",
        "for (int64_t I = 0; I < nc; I++) bc[I] = bc[I];",
        lambda o: T_prec.test_vcycle_rounding_points(o, 2, 32)),
    # the smoothing residual rounded to FP32 before it is used
    "extra rounding of the residual": (
        "x[i] = rnd(x[i] + dv[i] * r[i], pv);",
        "x[i] = rnd(x[i] + dv[i] * rnd(r[i], pv), pv);",
        lambda o: T_prec.test_vcycle_rounding_points(o, 2, 32)),
    # Dirichlet faces of the matrix with half the boundary transmissibility
    "Dirichlet factor": (
        "tb[s] = (F * (2.0 * ki)) / h;",
        "tb[s] = (F * ki) / h;",
        lambda o: T_asm.test_linear_field_exact_without_fractures(o, 2, 8)),
}


@pytest.fixture
def mutated_oracle(tmp_path, monkeypatch, oracle_mod):
    def make(old, new):
        src = open(oracle.SRC).read()
        assert old in src, "planted edit no longer matches the oracle source"
        d = tmp_path / "oracle"
        d.mkdir()
        (d / "mdoracle.c").write_text(src.replace(old, new, 1))
        shutil.copy(os.path.join(oracle.HERE, "mdoracle.h"), d / "mdoracle.h")
        lib = d / "liboracle.so"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib),
                               str(d / "mdoracle.c"), "-lm"])
        monkeypatch.setattr(oracle, "SRC", str(d / "mdoracle.c"))
        monkeypatch.setattr(oracle, "LIB", str(lib))
        monkeypatch.setattr(oracle, "_lib", None)  # restored to the real library afterwards
        return oracle
    return make


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_pin_catches_planted_mistake(mutated_oracle, name):
    old, new, pin = MUTATIONS[name]
    bad = mutated_oracle(old, new)
    with pytest.raises(AssertionError):
        pin(bad)


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_pin_passes_on_the_real_oracle(oracle_mod, name):
    MUTATIONS[name][2](oracle_mod)
