"""Mutation check of the oracle's pins (not collected by pytest).

Each mutant is one plausible mistake planted in a scratch copy of the
oracle.  In oracle/louvain_oracle.c: a dropped or sign-flipped term of
Eq. 2, a reversed tie-break or Pick-Less rule, a missing Sigma' or C'
update, a stopping rule off at its boundary, a missing dendrogram lookup,
and so on, and in its Leiden form a refinement that ignores P, lets chosen
vertices move or misstates the well-connectedness condition; the copy is
compiled and tests/test_oracle_pins.py and tests/test_oracle_leiden.py run
against it.  In oracle/mlp.py (the predictor): a missing ReLU or bias, a transposed
weight or gradient, a wrong loss scale or sign, bf16 rounding without ties
to even; tests/test_oracle_mlp.py runs against it.  Every mutant must make
some pin fail.  The repository's own oracle is never modified.

    python tests/oracle_mutants.py [scratch_dir]

Exit status 1 if a mutant survives."""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "score_own drops -K_i": ("(i128)K_i * (Sigma_d - K_i);", "(i128)K_i * Sigma_d;"),
    "score_other sign": ("return (i128)two_m * K_ic - (i128)K_i * Sigma_c;",
                         "return (i128)two_m * K_ic + (i128)K_i * Sigma_c;"),
    "tie-break to the highest id": ("(s == best_s && c < best_c)", "(s == best_s && c > best_c)"),
    "move on an equal score": ("!(best_s > s_d)", "!(best_s >= s_d)"),
    "pick-less direction": ("if (pickless && best_c > d) return out;", "if (pickless && best_c < d) return out;"),
    "pick-less phase": ("((li + rho / 2) % rho) == 0", "(li % rho) == 0"),
    "pick-less never": ("const int pickless = rho > 0 && ((li + rho / 2) % rho) == 0;", "const int pickless = 0;"),
    "self-loop in the move scan": ("if (!self && j == i) continue;", "if (0 && j == i) continue;"),
    "K_id ignored": ("    if (buf[t].c == d) K_id = buf[t].w;", "    if (0) K_id = buf[t].w;"),
    "no Sigma_d update": ("        Sigma[d] -= K[i];\n", ""),
    "no C' update": ("        Cp[i] = c;\n        dQ += dec[a].gain;", "        dQ += dec[a].gain;"),
    "gain not summed": ("        dQ += dec[a].gain;\n", ""),
    "no neighbour re-mark": ("if (g->col[e] != i) unprocessed[g->col[e]] = 1;", "if (0) unprocessed[g->col[e]] = 1;"),
    "evaluated not counted": ("      evaluated += na;\n", ""),
    "tau test without the factor 2": ("(double)(2 * dQ) / (double)den2", "(double)(dQ) / (double)den2"),
    "l_i off by one": ("if (total <= tau) { li_done = li + 1; break; }", "if (total <= tau) { li_done = li; break; }"),
    "aggregation drops self-loops": (
        "            buf[k].c = Cp[g->col[e]];\n            buf[k].w = g->w[e];\n            ++k;",
        "            if (g->col[e] == i) continue;\n            buf[k].c = Cp[g->col[e]];\n"
        "            buf[k].w = g->w[e];\n            ++k;"),
    "K without the self-loop": ("for (int64_t e = G.off[i]; e < G.off[i + 1]; ++e) s += G.w[e];",
                                "for (int64_t e = G.off[i]; e < G.off[i + 1]; ++e) if (G.col[e] != i) s += G.w[e];"),
    "m instead of 2m": ("  for (int64_t k = 0; k < G.nnz; ++k) two_m += G.w[k];\n",
                        "  for (int64_t k = 0; k < G.nnz; ++k) two_m += G.w[k];\n  two_m /= 2;\n"),
    "converged only at l_i < 1": ("if (li <= 1) { pending = 1;", "if (li < 1) { pending = 1;"),
    "aggregation tolerance >=": ("(double)nagg / (double)np > cfg->aggregation_tolerance",
                                 "(double)nagg / (double)np >= cfg->aggregation_tolerance"),
    "tau grows": ("tau /= cfg->tolerance_drop;", "tau *= cfg->tolerance_drop;"),
    "tau scaled before the first pass": ("  double tau = cfg->tolerance;",
                                         "  double tau = cfg->tolerance / cfg->tolerance_drop;"),
    "no dendrogram lookup": (
        "    for (int64_t v = 0; v < n; ++v) C[v] = agg[C[v]];                 /* dendrogram lookup */\n", ""),
    "no final lookup after a break": ("  if (pending)\n    for (int64_t v = 0; v < n; ++v) C[v] = Cp[C[v]];\n", ""),
    "renumbering reversed": ("  for (int64_t i = 0; i < len; ++i) x[i] = newid[x[i]];",
                             "  for (int64_t i = 0; i < len; ++i) x[i] = (int32_t)(run - 1 - newid[x[i]]);"),
    "S_in without self-loops": ("if (C[g->col[e]] == C[i]) s_in += g->w[e];",
                                "if (C[g->col[e]] == C[i] && g->col[e] != i) s_in += g->w[e];"),
    "S_tot not squared": ("s_tot += (i128)Sig[c] * Sig[c];", "s_tot += (i128)Sig[c];"),
    "bucket by mask": ("return fmix32((uint32_t)i ^ salt) % (uint32_t)B;",
                       "return fmix32((uint32_t)i ^ salt) & (uint32_t)(B - 1);"),
    # the Leiden form
    "refine ignores the communities of P": ("g->col[e] != i && bound[g->col[e]] == bound[i]", "g->col[e] != i"),
    "refine: chosen vertices still move": ("if (!dec[a].moves || chosen[v]) continue;", "if (!dec[a].moves) continue;"),
    "refine: well-connectedness reversed": ("elig[v] = (i128)two_m * kin >= ", "elig[v] = (i128)two_m * kin < "),
    "refine: well-connectedness without -K_v": ("(Sigma_b[bound[v]] - K[v]);", "Sigma_b[bound[v]];"),
    "refine: target total not updated": ("      Sr[t] += K[v];\n", ""),
    "Leiden: refinement over B buckets, not 4B": ("OR_REFINE_BUCKETS_PER_B * cfg->buckets", "cfg->buckets"),
    "Leiden: next pass from singletons": ("if (cfg->refine && lp > 0) {", "if (0) {"),
    "Leiden: pass cap returns the refinement": ("if (!pending && cfg->refine && passes > 0)", "if (0)"),
}


MLP_MUTANTS = {
    "no ReLU on the second layer": ('h2 = rb(np.maximum(z2, 0.0))', 'h2 = rb(z2)'),
    "no second-layer bias": ('z2 = h1 @ W2 + P["b2"]', 'z2 = h1 @ W2'),
    "W2 transposed": ('z2 = h1 @ W2 + P["b2"]', 'z2 = h1 @ W2.T + P["b2"]'),
    "loss gradient not divided by n": ('dl = (p - Y) / n', 'dl = (p - Y)'),
    "ReLU mask of the wrong layer": ('dz1 = dh1 * (c["z1"] > 0)', 'dz1 = dh1 * (c["z2"] > 0)'),
    "W2 gradient transposed": ('g["W2"] = c["h1"].T @ dz2b', 'g["W2"] = (c["h1"].T @ dz2b).T'),
    "back-propagation through W2, not its transpose": ('dh1 = dz2b @ c["W2"].T', 'dh1 = dz2b @ c["W2"]'),
    "bf16 rounds half up": ('+ np.uint64(0x7FFF) + lsb)', '+ np.uint64(0x8000))'),
    "loss sign": ('- logit * Y +', '+ logit * Y +'),
    "b3 gradient averaged": ('g["b3"] = dl.sum()', 'g["b3"] = dl.mean()'),
}


def copy_tree(scratch: str) -> str:
    for sub in ("oracle", os.path.join("paper_2501_19004_gb300", "graphgen"), os.path.join("tests", "golden")):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(scratch, sub), dirs_exist_ok=True,
                        ignore=shutil.ignore_patterns("__pycache__", "*.so"))
    for f in ("paper_2501_19004_gb300/__init__.py", "tests/conftest.py", "tests/test_oracle_pins.py",
              "tests/test_oracle_leiden.py", "tests/test_oracle_mlp.py"):
        shutil.copy(os.path.join(ROOT, f), os.path.join(scratch, f))
    return os.path.join(scratch, "oracle", "louvain_oracle.c")


def build_libs(scratch: str) -> None:
    sys.path.insert(0, scratch)
    subprocess.check_call([sys.executable, "-c", "import oracle; oracle.build(force=True); "
                           "from paper_2501_19004_gb300 import graphgen as gg; gg.build()"], cwd=scratch)


def main() -> int:
    scratch = sys.argv[1] if len(sys.argv) > 1 else tempfile.mkdtemp(prefix="oracle_mutants_")
    os.makedirs(scratch, exist_ok=True)
    src = copy_tree(scratch)
    build_libs(scratch)
    orig = open(src).read()
    lib = os.path.join(scratch, "oracle", "liblouvain_oracle.so")
    pins = [sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "tests/test_oracle_leiden.py", "-x", "-q",
            "-p", "no:cacheprovider"]
    assert subprocess.run(pins, cwd=scratch, capture_output=True).returncode == 0, "pins fail on the unmutated copy"
    survivors = 0
    try:
        for name, (old, new) in MUTANTS.items():
            assert orig.count(old) >= 1, f"mutant pattern not found: {name}"
            open(src, "w").write(orig.replace(old, new))
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", lib, src])
            r = subprocess.run(pins, cwd=scratch, capture_output=True, text=True, timeout=900)
            failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
            if r.returncode:
                print(f"{name:34s} killed by {failed[0].split('::')[1].split(' ')[0] if failed else '(error)'}")
            else:
                survivors += 1
                print(f"{name:34s} SURVIVED")
    finally:
        open(src, "w").write(orig)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", lib, src])
    mlp_src = os.path.join(scratch, "oracle", "mlp.py")
    mlp_orig = open(mlp_src).read()
    mlp_pins = [sys.executable, "-m", "pytest", "tests/test_oracle_mlp.py", "-x", "-q", "-p", "no:cacheprovider"]
    assert subprocess.run(mlp_pins, cwd=scratch, capture_output=True).returncode == 0, "MLP pins fail unmutated"
    try:
        for name, (old, new) in MLP_MUTANTS.items():
            assert mlp_orig.count(old) >= 1, f"mutant pattern not found: {name}"
            open(mlp_src, "w").write(mlp_orig.replace(old, new, 1))
            r = subprocess.run(mlp_pins, cwd=scratch, capture_output=True, text=True, timeout=900)
            failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
            if r.returncode:
                print(f"mlp: {name:48s} killed by {failed[0].split('::')[1].split(' ')[0] if failed else '(error)'}")
            else:
                survivors += 1
                print(f"mlp: {name:48s} SURVIVED")
    finally:
        open(mlp_src, "w").write(mlp_orig)
    total = len(MUTANTS) + len(MLP_MUTANTS)
    print(f"{total - survivors} of {total} mutants killed")
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main())
