"""Planted mistakes in the oracle: each one must fail at least one pin.

A pin that no plausible mistake can fail pins nothing.  Each case below plants
one mistake of the kind a transcription of the paper's method could make (a
dropped term, a wrong sign or index, a transposed operand, a swapped constant)
into a copy of the oracle's C source, builds it with the same gcc flags into a
temporary directory, and runs the pin tests that cover that routine against the
planted build (loaded through DQMC_ORACLE_LIB).  The run must report failing
tests (pytest exit status 1): a crash or a collection error does not count as
caught.  The unmodified source built the same way must pass the same pins, so a
failure comes from the plant and not from the harness.  The plants touch only
the temporary copy; the oracle on disk is never changed.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dqmc_oracle.c")

CORE = "tests/test_oracle_pins.py"
TAU = "tests/test_oracle_tau_pins.py"
CORR = "tests/test_oracle_corr_pins.py"
SU2 = "tests/test_oracle_su2_pins.py"
TAUC = "tests/test_oracle_tau_corr_pins.py"
SVD = "tests/test_oracle_svd_pins.py"
BOND = "tests/test_oracle_bond_ising_pins.py"

# (name, [(text in the source, its replacement), ...], the pins that must catch it)
PLANTS = [
    ("philox key schedule constant",
     [("k[1] += 0xBB67AE85u;", "k[1] += 0xBB67AE84u;")], [CORE + "::test_philox_known_answers"]),
    ("lambda from exp(dtau U / 4) (Ising coupling)",
     [("acosh(exp(0.5 * dtau * U))", "acosh(exp(0.25 * dtau * U))")], [CORE + "::test_ising_decoupling_is_exact"]),
    ("gamma values of the four-valued field swapped",
     [("if (l == 1 || l == -1) return 1.0 + s6 / 3.0;", "if (l == 1 || l == -1) return 1.0 - s6 / 3.0;"),
      ("if (l == 2 || l == -2) return 1.0 - s6 / 3.0;", "if (l == 2 || l == -2) return 1.0 + s6 / 3.0;")],
     [CORE + "::test_hs4_constants_match_paper_identity"]),
    ("B_tau^T applied as E^T on the outside (left chain order)",
     [("""  slice_potential(M, f, s, tau, v);
  mat_mul(N, M->ET + (size_t)s * N * N, X, X);
  for (int i = 0; i < N; ++i) {
    const double e = exp(v[i]);
    for (int j = 0; j < N; ++j) X[i * N + j] *= e;
  }""", """  slice_potential(M, f, s, tau, v);
  for (int i = 0; i < N; ++i) {
    const double e = exp(v[i]);
    for (int j = 0; j < N; ++j) X[i * N + j] *= e;
  }
  mat_mul(N, M->ET + (size_t)s * N * N, X, X);""")], [CORE + "::test_udv_agrees_with_plain_product"]),
    ("pivot permutation left out of T",
     [("u->T + (size_t)perm[k] * N", "u->T + (size_t)k * N")], [CORE + "::test_free_fermion_closed_form"]),
    ("D^-1 left out of T",
     [("Tn[i * N + j] = (Dn[i] > 0.0) ? acc / Dn[i] : 0.0;", "Tn[i * N + j] = acc;")], [CORE + "::test_free_fermion_closed_form"]),
    ("large and small scales swapped in the middle matrix",
     [("Mid[i * N + j] = QRtQL[i * N + j] / (dbR[i] * dbL[j]) + dsR[i] * TRTLt[i * N + j] * dsL[j];",
       "Mid[i * N + j] = QRtQL[i * N + j] / (dsR[i] * dsL[j]) + dbR[i] * TRTLt[i * N + j] * dbL[j];")], [CORE + "::test_free_fermion_closed_form"]),
    ("det Q of the left chain dropped from the sign",
     [("*sign = sm * R->detQ * Lf->detQ;", "*sign = sm * R->detQ;")], [CORE + "::test_udv_sign_per_flavor_odd_lattice"]),
    ("V-wrap with the wrong sign",
     [("*= exp(a * (v[x] - v[y]));", "*= exp(a * (v[y] - v[x]));")], [CORE + "::test_wrapped_sherman_morrison_matches_fresh"]),
    ("T-wrap with E and E^-1 exchanged on the way up",
     [("""    mat_mul(N, c->M.E + s * nn, c->G[s], c->G[s]);
    mat_mul(N, c->G[s], c->M.Einv + s * nn, c->G[s]);
  } else {""", """    mat_mul(N, c->M.Einv + s * nn, c->G[s], c->G[s]);
    mat_mul(N, c->G[s], c->M.E + s * nn, c->G[s]);
  } else {""")], [CORE + "::test_wrapped_sherman_morrison_matches_fresh"]),
    ("G_ii for 1 - G_ii in the ratio",
     [("Rs[s] = 1.0 + delta[s] * (1.0 - c->G[s][i * N + i]);", "Rs[s] = 1.0 + delta[s] * c->G[s][i * N + i];")],
     [CORE + "::test_wrapped_sherman_morrison_matches_fresh"]),
    ("gamma ratio inverted",
     [("double R = orc_field_gamma(M->ft, fn) / orc_field_gamma(M->ft, f);",
       "double R = orc_field_gamma(M->ft, f) / orc_field_gamma(M->ft, fn);")], [CORE + "::test_wrapped_sherman_morrison_matches_fresh"]),
    ("acceptance test inverted",
     [("if (u2 < (absR < 1.0 ? absR : 1.0)) {", "if (u2 > (absR < 1.0 ? absR : 1.0)) {")], [CORE + "::test_wrapped_sherman_morrison_matches_fresh"]),
    ("sign not flipped on a negative ratio",
     [("if (R < 0) c->sign = -c->sign;", "if (R < 0) c->sign = c->sign;")], [CORE + "::test_sign_tracked_through_negative_ratios"]),
    ("Sherman-Morrison row transposed",
     [("row[y] = ((y == i) ? 1.0 : 0.0) - G[i * N + y];", "row[y] = ((y == i) ? 1.0 : 0.0) - G[y * N + i];")],
     [CORE + "::test_wrapped_sherman_morrison_matches_fresh"]),
    ("kinetic energy with the wrong sign of G",
     [("kin += K[x * N + y] * ((x == y ? 1.0 : 0.0) - G[s][y * N + x]);",
       "kin += K[x * N + y] * ((x == y ? 1.0 : 0.0) + G[s][y * N + x]);")], [CORE + "::test_free_fermion_closed_form"]),
    ("potential energy at a shifted site",
     [("pot += M->U * (1.0 - G[0][i * N + i]) * (1.0 - G[1][i * N + i]);",
       "pot += M->U * (1.0 - G[0][i * N + i]) * (1.0 - G[1][((i + 1) % N) * (N + 1)]);")], [CORE + "::test_enumeration_equals_fock_trace_ising"]),
    ("d lambda / dU with cosh for sinh",
     [("/ sinh(lam) * (double)f;", "/ cosh(lam) * (double)f;")], [CORE + "::test_logdet_gradient_finite_differences"]),
    ("G(0,tau) with the wrong sign",
     [("G0t[i * N + j] = -acc;", "G0t[i * N + j] = acc;")], [TAU + "::test_displaced_green_antiperiodic_at_beta"]),
    ("G(tau,0) with the large scale of the right chain for the small one",
     [("acc += X[i * N + k] * (dR > 1.0 ? 1.0 : dR) * R->T[k * N + j];",
       "acc += X[i * N + k] * (dR > 1.0 ? dR : 1.0) * R->T[k * N + j];")], [CORE + "::test_displaced_green_against_plain_products"]),
    ("S^z S^z correlation with 1/2 for 1/4",
     [("out[c * 4 + 0] += 0.25 * (mx * my + X0 + X1);", "out[c * 4 + 0] += 0.5 * (mx * my + X0 + X1);")],
     [CORR + "::test_correlations_enumeration_equals_fock_trace"]),
    ("exchange term of n n with the wrong sign",
     [("out[c * 4 + 1] += rx * ry + X0 + X1;", "out[c * 4 + 1] += rx * ry - X0 - X1;")], [CORR + "::test_correlations_enumeration_equals_fock_trace"]),
    ("SU(2): phase of the bosonic factor with the wrong sign",
     [("hs_eta(fields[(size_t)(tau - 1) * N + x]);\n      ph -= th;",
       "hs_eta(fields[(size_t)(tau - 1) * N + x]);\n      ph += th;")], [SU2 + "::test_su2_enumeration_equals_fock_trace"]),
    ("SU(2): potential energy without the constant",
     [("pot += 0.5 * U * (2.0 * h * h - 2.0 * h + 1.0);", "pot += 0.5 * U * (2.0 * h * h - 2.0 * h);")], [SU2 + "::test_su2_enumeration_equals_fock_trace"]),
    ("S^z(tau) S^z(0): exchange term with the wrong sign",
     [("const double X0 = -G0t[0][y * N + x] * Gt0[0][x * N + y];",
       "const double X0 = G0t[0][y * N + x] * Gt0[0][x * N + y];")], [TAUC + "::test_enumeration_equals_fock_trace"]),
    ("time-displaced Green function per class transposed",
     [("o[0] += Gt0[0][x * N + y] + Gt0[1][x * N + y];", "o[0] += Gt0[0][y * N + x] + Gt0[1][y * N + x];")],
     [TAUC + "::test_single_configuration_against_plain_products"]),
    ("n(tau) n(0): the density at time 0 taken at tau",
     [("const double nyu = 1.0 - G00[0][y * N + y], nyd = 1.0 - G00[1][y * N + y];",
       "const double nyu = 1.0 - Gtt[0][y * N + y], nyd = 1.0 - Gtt[1][y * N + y];")], [TAUC + "::test_single_configuration_against_plain_products"]),
    ("SVD chain: T updated with V for V^T",
     [("acc += V[k * N + i] * u->T[k * N + j];", "acc += V[i * N + k] * u->T[k * N + j];")], [SVD + "::test_svd_chain_equals_plain_product"]),
    ("SVD chain: squared singular values as D",
     [("S[j] = sqrt(s2);", "S[j] = s2;")], [SVD + "::test_svd_chain_equals_plain_product"]),
    ("SU(2) UDV chain: pi of a negative det Q_R det Q_L dropped",
     [("if (R->detQ * Lf->detQ < 0) ar += 3.14159265358979323846;",
       "if (0) ar += 3.14159265358979323846;")], [SU2 + "::test_su2_udv_chain_matches_plain_product"]),
    ("SU(2) UDV chain: T_L^T for T_L^H in the middle matrix",
     [("conj(Lf->T[(size_t)j * N + k]);   /* T_R T_L^H */", "Lf->T[(size_t)j * N + k];   /* T_R T_L^H */")],
     [SU2 + "::test_su2_udv_chain_matches_plain_product"]),
    ("bond model: bond factors applied in the reverse order",
     [("for (int b = nb - 1; b >= 0; --b) {\n      const double a = -dtau * xi",
       "for (int b = 0; b < nb; ++b) {\n      const double a = -dtau * xi")], [BOND + "::test_enumeration_equals_trotter_trace_two_bonds_interacting"]),
    ("bond model: sinh with the wrong sign in the plain product",
     [("B[(size_t)i * N + y] = ch * ri + sh * rj;", "B[(size_t)i * N + y] = ch * ri - sh * rj;"),
      ("B[(size_t)j * N + y] = sh * ri + ch * rj;", "B[(size_t)j * N + y] = -sh * ri + ch * rj;")], [BOND + "::test_vertex_green_ratios_and_rank2_update"]),
    ("bond model: HS phase dropped from the plain product",
     [("hs_eta(hs[(size_t)(tau - 1) * N + x]);\n      ph -= th;", "hs_eta(hs[(size_t)(tau - 1) * N + x]);\n      ph -= 0.0;")],
     [BOND + "::test_enumeration_equals_trotter_trace_interacting"]),
    ("bond spins: cosh and sinh of the transverse field swapped",
     [("(s[b] == sn[b]) ? log(cosh(dtau * h)) : log(sinh(dtau * h));",
       "(s[b] == sn[b]) ? log(sinh(dtau * h)) : log(cosh(dtau * h));")], [BOND + "::test_enumeration_equals_trotter_trace_two_bonds_free_fermions"]),
    ("bond spins: open boundary in imaginary time",
     [("for (int b = 0; b < nb; ++b) lw += (s[b] == sn[b])", "for (int b = 0; b < nb && tau + 1 < L; ++b) lw += (s[b] == sn[b])")],
     [BOND + "::test_enumeration_equals_trotter_trace_two_bonds_free_fermions"]),
    ("bond flip: determinant ratio not squared (one color)",
     [("R = rf * rf * exp(lw1 - lw0);", "R = rf * exp(lw1 - lw0);")], [BOND + "::test_sampler_matches_trotter_product"]),
    ("bond flip: bond spins' weight ratio inverted",
     [("R = rf * rf * exp(lw1 - lw0);", "R = rf * rf * exp(lw0 - lw1);")], [BOND + "::test_sampler_matches_trotter_product"]),
    ("rank-2 update: rows of G for rows of 1 - G",
     [("R[(size_t)a * N + y] = (P[a] == y ? 1.0 : 0.0) - GC(P[a], y);", "R[(size_t)a * N + y] = GC(P[a], y);")],
     [BOND + "::test_rank2_update_with_a_general_delta"]),
    ("rank-2 update: delta transposed",
     [("Wm[2 * a + b] = Si[2 * a] * d[b] + Si[2 * a + 1] * d[2 + b];",
       "Wm[2 * a + b] = Si[2 * a] * d[2 * b] + Si[2 * a + 1] * d[2 * b + 1];")], [BOND + "::test_rank2_update_with_a_general_delta"]),
    ('53-bit uniform from 52 bits',
     [('return (double)(w >> 11) * (1.0 / 9007199254740992.0);', 'return (double)(w >> 12) * (1.0 / 9007199254740992.0);')],
     [CORE + "::test_uniform_mapping"]),
    ('initial four-valued fields drawn from three values',
     [('int idx = (int)floor(4.0 * u);', 'int idx = (int)floor(3.0 * u);')],
     [CORE + "::test_init_fields_distribution"]),
    ('four-valued proposal restricted to two of the three other values',
     [('int idx = (int)floor(3.0 * u1);\n    if (idx > 2) idx = 2;\n    fn = others[idx];', 'int idx = (int)floor(2.0 * u1);\n    if (idx > 2) idx = 2;\n    fn = others[idx];')],
     [CORE + "::test_sampler_reproduces_exact_energies"]),
    ('LU: sign of a negative pivot ignored',
     [('    if (d < 0) sg = -sg;\n', '')],
     [CORE + "::test_logdet_against_library"]),
    ('Jacobi rotation with the wrong sign of s',
     [('const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;', 'const double c = 1.0 / sqrt(t * t + 1.0), s = -t * c;')],
     [CORE + "::test_eig_and_expm_against_library"]),
    ('log-det adjoint: V-wrap of G(tau-1) with the wrong sign',
     [('- exp(v[x] - v[y]) * G[x * N + y];', '- exp(v[y] - v[x]) * G[x * N + y];')],
     [CORE + "::test_logdet_gradient_finite_differences"]),
    ('log-det adjoint: E for E^-1',
     [('mat_mul(N, S, M.Einv + s * nn, A);', 'mat_mul(N, S, M.E + s * nn, A);')],
     [CORE + "::test_logdet_gradient_finite_differences"]),
    ('energy adjoint: explicit delta - G^T term dropped on the diagonal',
     [('if (x == y) g[x * N + y] = Z[x * N + y] + ex;', 'if (x == y) g[x * N + y] = Z[x * N + y];')],
     [CORE + "::test_energy_gradient_finite_differences"]),
    ('energy adjoint: divided difference sinh(x) for sinh(x)/x',
     [('const double x = 0.5 * M.dtau * (w[a] - w[b]);\n          const double shc = (x == 0.0) ? 1.0 : sinh(x) / x;', 'const double x = 0.5 * M.dtau * (w[a] - w[b]);\n          const double shc = (x == 0.0) ? 1.0 : sinh(x);')],
     [CORE + "::test_energy_gradient_finite_differences"]),
    ("energy adjoint: the own flavor's density in dPot/dK_xx",
     [('g -= M.U * (1.0 - G0[1 - s][x * N + x]);', 'g -= M.U * (1.0 - G0[s][x * N + x]);')],
     [CORE + "::test_energy_gradient_finite_differences"]),
    ('tau observables: connected density term with the wrong sign',
     [('c -= px * py * G0t[y * N + x] * Gt0[x * N + y];', 'c += px * py * G0t[y * N + x] * Gt0[x * N + y];')],
     [TAU]),
    ('tau observables: density at tau taken from G(tau,0)',
     [('p += px * (1.0 - Gtt[x * N + x]);', 'p += px * (1.0 - Gt0[x * N + x]);')],
     [TAU]),
    ('SU(2) correlations: S^z S^z with 1/4 X for 1/2 X',
     [('const double complex v[4] = {0.5 * X, rx * ry + 2.0 * X, X, 2.0 * hyx};', 'const double complex v[4] = {0.25 * X, rx * ry + 2.0 * X, X, 2.0 * hyx};')],
     [SU2 + "::test_su2_correlations_enumeration_equals_fock_trace"]),
    ('SU(2) left chain: e^{V} for its adjoint e^{-V}',
     [('const double complex ev = cexp(-_Complex_I * g * hs_eta(fields[(size_t)(t - 1) * N + x]));', 'const double complex ev = cexp(_Complex_I * g * hs_eta(fields[(size_t)(t - 1) * N + x]));')],
     [SU2 + "::test_su2_udv_chain_matches_plain_product"]),
    ('SU(2) G(0,tau) with the wrong sign',
     [('G0t[2 * ((size_t)i * N + j)] = -creal(acc);\n        G0t[2 * ((size_t)i * N + j) + 1] = -cimag(acc);', 'G0t[2 * ((size_t)i * N + j)] = creal(acc);\n        G0t[2 * ((size_t)i * N + j) + 1] = cimag(acc);')],
     [SU2 + "::test_su2_displaced_green_matches_the_definition"]),
    ('SU(2) G(tau,0) with Db_R for Ds_R',
     [('X[(size_t)i * N + j] = MI[(size_t)i * N + j] / dbL[i] * dsR[j];', 'X[(size_t)i * N + j] = MI[(size_t)i * N + j] / dbL[i] * dbR[j];')],
     [SU2 + "::test_su2_displaced_green_matches_the_definition"]),
    ('SU(2) acceptance with |R| instead of the phase-reweighted |Re(P R)| / |Re P|',
     [('const double ratio = fabs(creal(P * R)) / fabs(creal(P));', 'const double ratio = cabs(R);')],
     [SU2 + "::test_su2_sweep_equals_brute_force_metropolis_on_full_weights"]),
    ('SU(2) initial phase with arg det for 2 arg det (one color)',
     [('P = cexp(_Complex_I * (ph + 2.0 * ar));   /* prod', 'P = cexp(_Complex_I * (ph + ar));   /* prod')],
     [SU2 + "::test_su2_phase_carried_equals_recomputed"]),
    ('bond model: site ratio not squared (one color)',
     [('          R = hs_gamma(fn) / hs_gamma(f) * cexp(-_Complex_I * dth) * r1 * r1;', '          R = hs_gamma(fn) / hs_gamma(f) * cexp(-_Complex_I * dth) * r1;')],
     [BOND + "::test_sampler_matches_trotter_product"]),
    ('bond flip: delta of the flip from a for 2a',
     [('const double delta[8] = {cosh(2.0 * a) - 1.0, 0.0, -sinh(2.0 * a), 0.0,\n                                   -sinh(2.0 * a), 0.0, cosh(2.0 * a) - 1.0, 0.0};', 'const double delta[8] = {cosh(a) - 1.0, 0.0, -sinh(a), 0.0,\n                                   -sinh(a), 0.0, cosh(a) - 1.0, 0.0};')],
     [BOND + "::test_sampler_matches_trotter_product"]),
    ('n(tau) n(0): exchange term with the wrong sign',
     [('o[2] += (nxu + nxd) * (nyu + nyd) + X0 + X1;', 'o[2] += (nxu + nxd) * (nyu + nyd) - X0 - X1;')],
     [TAUC + "::test_enumeration_equals_fock_trace"]),
    ("SU(2) n n correlation with one color's exchange term",
     [('const double complex v[4] = {0.5 * X, rx * ry + 2.0 * X, X, 2.0 * hyx};', 'const double complex v[4] = {0.5 * X, rx * ry + X, X, 2.0 * hyx};')],
     [SU2 + "::test_su2_correlations_enumeration_equals_fock_trace"]),
    ('four-valued eta(2) equal to eta(1)',
     [('case 2: return sqrt(2.0 * (3.0 + s6));', 'case 2: return sqrt(2.0 * (3.0 - s6));')],
     [CORE + "::test_hs4_constants_match_paper_identity"]),
    ('B_tau = e^V E instead of E e^V (equal-time G shifted by a similarity)',
     [('  slice_potential(M, f, s, tau, v);\n  for (int i = 0; i < N; ++i) {\n    const double e = exp(v[i]);\n    for (int j = 0; j < N; ++j) X[i * N + j] *= e;\n  }\n  mat_mul(N, M->E + (size_t)s * N * N, X, X);', '  slice_potential(M, f, s, tau, v);\n  mat_mul(N, M->E + (size_t)s * N * N, X, X);\n  for (int i = 0; i < N; ++i) {\n    const double e = exp(v[i]);\n    for (int j = 0; j < N; ++j) X[i * N + j] *= e;\n  }')],
     [TAU + "::test_tau_enumeration_equals_fock_trace"]),
    ('complex Householder reflection without the conjugate',
     [('for (int i = k; i < N; ++i) s += conj(v[i]) * X[(size_t)i * N + j];', 'for (int i = k; i < N; ++i) s += v[i] * X[(size_t)i * N + j];')],
     [SU2 + "::test_su2_udv_chain_matches_plain_product"]),
    ('complex QR: reflections not counted in det Q',
     [('betas[k] = 2.0 / vhv;\n    dq = -dq;', 'betas[k] = 2.0 / vhv;')],
     [SU2 + "::test_su2_udv_chain_matches_plain_product"]),
    ('complex chain: pivot permutation left out of T',
     [('acc += X[(size_t)i * N + k] * u->T[(size_t)perm[k] * N + j];', 'acc += X[(size_t)i * N + k] * u->T[(size_t)k * N + j];')],
     [SU2 + "::test_su2_udv_chain_matches_plain_product"]),
    ("stable G(tau): the right chain's last chunk overshoots tau",
     [('  for (int t = 0; t < tau; t += nw) udv_right_step(&M, fields, s, t, (t + nw < tau) ? t + nw : tau, &R);\n  for (int t = M.L; t > tau; t -= nw) udv_left_step(&M, fields, s, (t - nw > tau) ? t - nw : tau, t, &Lf);\n  st = green_from_udv(', '  for (int t = 0; t < tau; t += nw) udv_right_step(&M, fields, s, t, t + nw, &R);\n  for (int t = M.L; t > tau; t -= nw) udv_left_step(&M, fields, s, (t - nw > tau) ? t - nw : tau, t, &Lf);\n  st = green_from_udv(')],
     [CORE + "::test_udv_agrees_with_plain_product"]),
    ("stable G(tau): the left chain's last chunk stops short of tau",
     [('  for (int t = 0; t < tau; t += nw) udv_right_step(&M, fields, s, t, (t + nw < tau) ? t + nw : tau, &R);\n  for (int t = M.L; t > tau; t -= nw) udv_left_step(&M, fields, s, (t - nw > tau) ? t - nw : tau, t, &Lf);\n  st = green_from_udv(', '  for (int t = 0; t < tau; t += nw) udv_right_step(&M, fields, s, t, (t + nw < tau) ? t + nw : tau, &R);\n  for (int t = M.L; t > tau; t -= nw) udv_left_step(&M, fields, s, (t - nw > tau) ? t - nw : tau + 1, t, &Lf);\n  st = green_from_udv(')],
     [CORE + "::test_udv_agrees_with_plain_product"]),
    ('S^+_x S^-_y with x and y exchanged',
     [('out[c * 4 + 2] += (dxy - G0[y * N + x]) * G1[x * N + y];', 'out[c * 4 + 2] += (dxy - G0[x * N + y]) * G1[y * N + x];')],
     [CORR + "::test_single_configuration_per_ordered_pair_equals_fock_trace"]),
    ('SU(2) correlations with x and y exchanged',
     [('      const double complex hyx = dxy - GZ(y, x);\n      const double complex X = hyx * GZ(x, y);', '      const double complex hyx = dxy - GZ(x, y);\n      const double complex X = hyx * GZ(y, x);')],
     [SU2 + "::test_su2_single_configuration_per_ordered_pair_equals_fock_trace"]),
    ('bond model left chain: e^{V} for its adjoint',
     [('          const double complex ev = cexp(-_Complex_I * m->g * hs_eta(m->hs[(size_t)(t - 1) * N + x]));', '          const double complex ev = cexp(_Complex_I * m->g * hs_eta(m->hs[(size_t)(t - 1) * N + x]));')],
     [BOND]),
    ("bond model left chain: factors in the right chain's order",
     [('      const int part = left ? m->nb + 1 - q : q;', '      const int part = q;')],
     [BOND]),
    ('log-det adjoint dU with G_ii for 1 - G_ii',
     [('        gU += (1.0 - G[i * N + i]) * M.sgn[s * M.MV + k] *', '        gU += G[i * N + i] * M.sgn[s * M.MV + k] *')],
     [CORE + "::test_logdet_gradient_finite_differences"]),
    ('energy adjoint dU without the flavor sign sigma_s',
     [('          gu += acc * M.sgn[s * M.MV + k] *', '          gu += acc *')],
     [CORE + "::test_energy_gradient_finite_differences"]),
    ('particle number from G_ii for 1 - G_ii',
     [('    for (int i = 0; i < N; ++i) part += 1.0 - G[s][i * N + i];', '    for (int i = 0; i < N; ++i) part += G[s][i * N + i];')],
     [CORE]),
    ('local G(tau) from G(0,tau) for G(tau,0)',
     [('        a += Gt0[x * N + x];', '        a += G0t[x * N + x];')],
     [TAU]),
    ('measurements not weighted by the sign',
     [('for (int q = 0; q < 4; ++q) c->meas[q] += (double)c->sign * e[q];', 'for (int q = 0; q < 4; ++q) c->meas[q] += e[q];')],
     [CORE + "::test_sampler_with_negative_weights_matches_exact_energies"]),
    ('ratio without the flavor sign sigma_s',
     [('delta[s] = exp(M->sgn[s * M->MV + k] * dc) - 1.0;', 'delta[s] = exp(dc) - 1.0;')],
     [CORE + "::test_wrapped_sherman_morrison_matches_fresh"]),
    ('V-unwrap of the down pass with the up sign',
     [('    for (int s = 0; s < nfl; ++s) v_wrap(c, s, tau, -1.0);', '    for (int s = 0; s < nfl; ++s) v_wrap(c, s, tau, +1.0);')],
     [CORE + "::test_wrapped_sherman_morrison_matches_fresh"]),
    ('up-pass stabilisation with the left chain of the previous point',
     [('        fresh_replace(c, s, &chain, (j == nst) ? &ident : &c->slot[s][j], &fs);', '        fresh_replace(c, s, &chain, (j == nst) ? &ident : &c->slot[s][j - 1], &fs);')],
     [CORE + "::test_free_fermion_closed_form"]),
    ('down-pass stabilisation from the wrong stored slot',
     [('        udv_copy(N, (j + 1 == nst) ? &ident : &c->slot[s][j + 1], &chain);', '        udv_copy(N, (j + 1 == nst) ? &ident : &c->slot[s][j], &chain);')],
     [CORE + "::test_free_fermion_closed_form"]),
    ('bond model: initial phase with one arg det',
     [('    P = cexp(_Complex_I * (ph + 2.0 * ar));\n  }\n  int acc = 0;\n  const int nv', '    P = cexp(_Complex_I * (ph + ar));\n  }\n  int acc = 0;\n  const int nv')],
     [BOND + "::test_sweep_equals_brute_force_metropolis_on_full_weights"]),
    ('bond model: site acceptance without the phase reweighting',
     [('          R = hs_gamma(fn) / hs_gamma(f) * cexp(-_Complex_I * dth) * r1 * r1;\n          const double rr = fabs(creal(P * R)) / fabs(creal(P));', '          R = hs_gamma(fn) / hs_gamma(f) * cexp(-_Complex_I * dth) * r1 * r1;\n          const double rr = cabs(R);')],
     [BOND + "::test_sweep_equals_brute_force_metropolis_on_full_weights"]),
    ('bond model: bond acceptance without the phase reweighting',
     [('          R = rf * rf * exp(lw1 - lw0);\n          const double rr = fabs(creal(P * R)) / fabs(creal(P));', '          R = rf * rf * exp(lw1 - lw0);\n          const double rr = cabs(R);')],
     [BOND + "::test_sweep_equals_brute_force_metropolis_on_full_weights"]),
    ('bond spins: J coupling with the wrong sign',
     [('lw += dtau * J * (double)(s[pairs[2 * q]] * s[pairs[2 * q + 1]]);', 'lw -= dtau * J * (double)(s[pairs[2 * q]] * s[pairs[2 * q + 1]]);')],
     [BOND + "::test_enumeration_equals_trotter_trace_two_bonds_interacting"]),
    ('bond factor of part p taken as bond p',
     [('    const int b = m->nb - part;', '    const int b = part - 1;')],
     [BOND]),
    ('Green function seen by a factor taken before it acts',
     [('  const int f = (tau - 1) * P + part;', '  const int f = (tau - 1) * P + part - 1;')],
     [BOND]),
    ('bond model: site ratio with G_xx for 1 - G_xx',
     [('          const double complex r1 = 1.0 + (cexp(_Complex_I * dth) - 1.0) * (1.0 - Gt[(size_t)x * N + x]);', '          const double complex r1 = 1.0 + (cexp(_Complex_I * dth) - 1.0) * Gt[(size_t)x * N + x];')],
     [BOND]),
]


def _build(directory: str, source: str) -> str:
    c = os.path.join(directory, "dqmc_oracle.c")
    with open(c, "w") as fh:
        fh.write(source)
    so = os.path.join(directory, "liboracle.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", so, c, "-lm"])
    return so


def _run_pins(lib: str, pins) -> int:
    env = dict(os.environ, DQMC_ORACLE_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", *pins, "-q", "-x", "-m", "not gpu", "-p", "no:cacheprovider"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900).returncode


def _planted_source(edits) -> str:
    with open(SRC) as fh:
        src = fh.read()
    for old, new in edits:
        assert src.count(old) == 1, f"the text to replace must occur exactly once: {old!r}"
        src = src.replace(old, new)
    return src


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """pytest status of the pins against every planted build and against the
    unplanted one ("control"), run concurrently (each in its own process)."""
    jobs = [("control", _planted_source([]), sorted({t for _, _, ts in PLANTS for t in ts}))]
    jobs += [(name, _planted_source(edits), pins) for name, edits, pins in PLANTS]

    base = tmp_path_factory.mktemp("plants")

    def run(job):
        k, (name, src, pins) = job
        d = os.path.join(str(base), f"plant{k}")
        os.makedirs(d)
        return name, _run_pins(_build(d, src), pins)

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(ex.map(run, enumerate(jobs)))


def test_unplanted_build_passes_the_pins(outcomes):
    assert outcomes["control"] == 0


@pytest.mark.parametrize("name,edits,pins", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_mistake_fails_a_pin(outcomes, name, edits, pins):
    assert outcomes[name] == 1, f"planted mistake '{name}' not caught by {pins} (pytest status {outcomes[name]})"
