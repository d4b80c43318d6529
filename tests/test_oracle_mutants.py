"""The oracle's pins must catch plausible mistakes.  Each case plants one mistake
(a dropped term, a wrong sign, a transposed operand, a wrong index or threshold) in
a temporary copy of the oracle source, builds it, and runs the pin tests against
it: they must fail.  CPU only; nothing here touches the product code."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gs_oracle.c")

MUTANTS = {
    "no_dilation": ("#define DILATION 0.3", "#define DILATION 0.0"),
    "jacobian_sign": ("J[0][2] = -fx * pr[P_RX] / z", "J[0][2] = fx * pr[P_RX] / z"),
    "transposed_rotation": ("T[i][j] = J[i][0] * R[0 * 3 + j] + J[i][1] * R[1 * 3 + j] + J[i][2] * R[2 * 3 + j];\n        cov6_to_mat(cov3d + 6 * (size_t)g, S);\n        for",
                            "T[i][j] = J[i][0] * R[j * 3 + 0] + J[i][1] * R[j * 3 + 1] + J[i][2] * R[j * 3 + 2];\n        cov6_to_mat(cov3d + 6 * (size_t)g, S);\n        for"),
    "q_cross_term": ("2.0 * pr[P_CB] * dx * dy", "pr[P_CB] * dx * dy"),
    "transmittance_update": ("T = test_T;", "T = T * c.alpha;"),
    "stop_rule": ("if (test_T < T_STOP) break;", "if (T < T_STOP) break;"),
    "clamp_value": ("#define ALPHA_CLAMP 0.99", "#define ALPHA_CLAMP 0.999"),
    "depth_order": ("if (x->zf < y->zf) return -1;\n    if (x->zf > y->zf) return 1;",
                    "if (x->zf < y->zf) return 1;\n    if (x->zf > y->zf) return -1;"),
    "topk_ascending": ("if (!taken[i] && (best < 0 || c[i].w > c[best].w)) best = i;",
                       "if (!taken[i] && (best < 0 || c[i].w < c[best].w)) best = i;"),
    "no_renormalisation": ("double wp = walk[pos[k]].w / S;", "double wp = walk[pos[k]].w;"),
    "u_uses_cy": ("pr[P_U] = cam[CAM_FX] * p[0] / p[2] + cam[CAM_CX];", "pr[P_U] = cam[CAM_FX] * p[0] / p[2] + cam[CAM_CY];"),
    "bwd_suffix_sign": ("- suffix / (1.0 - c->alpha)", "+ suffix / (1.0 - c->alpha)"),
    "bwd_conic_b_factor": ("dq * 2.0 * c->dx * c->dy", "dq * c->dx * c->dy"),
    "bwd_mean2d_sign": ("dq * -2.0 * (pr[P_CA] * c->dx", "dq * 2.0 * (pr[P_CA] * c->dx"),
    "bwd_rgb_uses_alpha": ("c->w * dCp[ch]", "c->alpha * dCp[ch]"),
    "bwd_dT_factor": ("dT[i][j] = 2.0 * acc;", "dT[i][j] = acc;"),
    "bwd_feature_term": ("acc += dFp[d] * (f[d] - Fp[d]);", "acc += dFp[d] * f[d];"),
    "bwd_jacobian_z": ("dpz += dJ[0][0] * (-fx / (z * z));", "dpz += dJ[0][0] * (fx / (z * z));"),
    "prune_counts_all_contributors": ("for (int k = 0; k < m; ++k) count[walk[pos[k]].g] += 1;",
                                      "for (int k = 0; k < nc; ++k) count[walk[k].g] += 1;"),
    "pose_no_covariance_term": ("g_view[4 * i + j] += dp[i] * mu[j] + J[0][i] * dT[0][j] + J[1][i] * dT[1][j];",
                                "g_view[4 * i + j] += dp[i] * mu[j];"),
    "pose_translation_sign": ("g_view[4 * i + 3] += dp[i];", "g_view[4 * i + 3] -= dp[i];"),
    "vanilla_uses_alpha": ("for (int d = 0; d < D; ++d) Fp[d] += walk[i].w * f[d];",
                           "for (int d = 0; d < D; ++d) Fp[d] += walk[i].alpha * f[d];"),
    "loss_grad_sign": ("(cosv * f[d] / ff - g[d] / (nf * ng))", "(g[d] / (nf * ng) - cosv * f[d] / ff)"),
    "loss_grad_norm_not_squared": ("cosv * f[d] / ff", "cosv * f[d] / nf"),
    "loss_rgb_not_averaged": ("w_rgb * l1c / 3.0", "w_rgb * l1c"),
    "loss_drgb_factor": ("dC[3 * p + i] = w_rgb * inv / 3.0 * sgn(e);", "dC[3 * p + i] = w_rgb * inv * sgn(e);"),
    "loss_not_a_mean": ("*loss = sum * inv;", "*loss = sum;"),
    "loss_zero_row_adds_nothing": ("sum += w_feat * (1.0 - cosv)",
                                   "sum += w_feat * (ff > 0.0 && gg > 0.0 ? 1.0 - cosv : 0.0)"),
    "loss_depth_sign": ("dD[p] = w_depth * inv * sgn(ed);", "dD[p] = -w_depth * inv * sgn(ed);"),
    "prune_importance_is_alpha": ("if (walk[i].w > maxw[walk[i].g]) maxw[walk[i].g] = walk[i].w;",
                                  "if (walk[i].alpha > maxw[walk[i].g]) maxw[walk[i].g] = walk[i].alpha;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    src = src.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "mut.c")
        so = os.path.join(td, "libmut.so")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", c, "-o", so, "-lm"])
        env = dict(os.environ, GS_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                            os.path.join(ROOT, "tests", "test_oracle_prune.py"),
                            os.path.join(ROOT, "tests", "test_oracle_loss.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
