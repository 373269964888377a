"""Planted mistakes in the oracles (CPU only), for the mutation test: each entry rewrites one line
of one oracle function, and the pins must catch every such mutant. Loaded as a pytest plugin
(-p oracle_mutants) in a child process; it changes nothing unless RTCUR_ORACLE_MUTANT names a
mutant."""
import importlib
import inspect
import os
import textwrap

# name: (module, function, original text, mutated text)
MUTANTS = {
    # forward oracle
    "ht_not_strict": ("oracle.rtcur_oracle", "hard_threshold", "np.abs(D) > zeta", "np.abs(D) >= zeta"),
    "pinv_s_inverted": ("oracle.rtcur_oracle", "truncated_pinv", "(V / s[None, :])", "(V * s[None, :])"),
    "err_squared_norms": ("oracle.rtcur_oracle", "relative_error",
                          "num = np.linalg.norm(ER) + sum(np.linalg.norm(E) for E in EC)",
                          "num = np.linalg.norm(ER) ** 2 + sum(np.linalg.norm(E) ** 2 for E in EC)"),
    "j_decode_reversed": ("oracle.rtcur_oracle", "other_mode_coords", "for l in reversed(range(len(dims))):",
                          "for l in range(len(dims)):"),
    "no_zeta_decay": ("oracle.rtcur_oracle", "rtcur", "zeta = gamma * zeta", "zeta = zeta"),
    "svd_keeps_r_plus_1": ("oracle.rtcur_oracle", "svd_truncated", "k = int(min(r, np.count_nonzero(s > tau)))",
                           "k = int(min(r + 1, np.count_nonzero(s > tau)))"),
    "s_sign_in_r": ("oracle.rtcur_oracle", "rtcur_step", "R = XR - SR", "R = XR + SR"),
    # adjoint oracle
    "adj_factor_2": ("oracle.rtcur_adjoint", "pinv_vjp", "Z @ Pbar.T + 2.0 * Mb @ W", "Z @ Pbar.T + 1.0 * Mb @ W"),
    "adj_coupling_dropped": ("oracle.rtcur_adjoint", "pinv_vjp", "F[j, k] = 1.0 / (lam[j] * (lam[j] - lam[k]))",
                             "F[j, k] = 0.0"),
    "adj_masks_inverted": ("oracle.rtcur_adjoint", "rtcur_vjp", 'np.where(t["mR"], 0.0, Rb)',
                           'np.where(t["mR"], Rb, 0.0)'),
    "adj_fiber_term_missing": ("oracle.rtcur_adjoint", "_eval_vjp", "Ab[i] += LbC[i] @ Z.T",
                               "Ab[i] += 0.0 * (LbC[i] @ Z.T)"),
    "adj_sign_flip": ("oracle.rtcur_adjoint", "rtcur_vjp", "cb = Ab[i] @ P.T", "cb = -(Ab[i] @ P.T)"),
}


def apply(name):
    modname, fname, old, new = MUTANTS[name]
    mod = importlib.import_module(modname)
    src = textwrap.dedent(inspect.getsource(getattr(mod, fname)))
    if old not in src:
        raise RuntimeError(f"mutant {name}: text not found in {modname}.{fname}")
    ns = dict(vars(mod))
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)
    setattr(mod, fname, ns[fname])


def pytest_configure(config):
    name = os.environ.get("RTCUR_ORACLE_MUTANT")
    if name:
        apply(name)
