"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the oracle pins catch every one: a dropped term, a wrong sign, a wrong
index, a wrong normalisation or exponent."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("G3 sign", "G3 = 2.0 * Phi * a[None, :] + np.outer(m1, nrm2)",
     "G3 = 2.0 * Phi * a[None, :] - np.outer(m1, nrm2)"),
    ("G2 pair factor", "G2 = U.T @ (Q * (2.0 * c * Q - 2.0 * H))",
     "G2 = U.T @ (Q * (1.0 * c * Q - 2.0 * H))"),
    ("R dropped", "G1 = X.T @ (Y * Y - R)", "G1 = X.T @ (Y * Y)"),
    ("alpha0 term of M3", "return (c3 * E3w - alpha0 * (alpha0 + 1.0) / 2.0 * perm3(E2w, m1)",
     "return (c3 * E3w - alpha0 * (alpha0 + 2.0) / 2.0 * perm3(E2w, m1)"),
    ("perm3 placement", 'np.einsum("il,j->ijl", Mat, v)', 'np.einsum("ij,l->ijl", Mat, v)'),
    ("m1^3 coefficient", "return c3 * C3 + perm3(np.eye(k), m1) - 2.0 * sym3(m1, m1, m1)",
     "return c3 * C3 + perm3(np.eye(k), m1) - 1.0 * sym3(m1, m1, m1)"),
    ("X not centred",
     'X = F @ W - st["L"][:, None].astype(np.float64) * m1[None, :]        # a2',
     "X = F @ W        # a2"),
    ("whitening exponent", "W = vec / np.sqrt(lam)[None, :]", "W = vec / lam[None, :]"),
    ("unwhitening power", "mu = pinv_transpose(W) @ (Phi * (n ** 2)[None, :])",
     "mu = pinv_transpose(W) @ (Phi * (n ** 3)[None, :])"),
    ("pair normalisation", "return (alpha0 + 1.0) * (P.astype(np.float64) / float(S2))",
     "return (alpha0 + 1.0) * (P.astype(np.float64) / float(S2 + 1000))"),
    ("Y from uncentred W", "Y = X @ Phi  ", "Y = (F @ W) @ Phi  "),
    ("sketch keeps the diagonal", "return F.T @ S - c[:, None] * Omega", "return F.T @ S"),
    ("sketched M2 rank-one sign", "Y = (alpha0 + 1.0) / float(S2) * Z - alpha0 * np.outer(M1, M1 @ Omega)",
     "Y = (alpha0 + 1.0) / float(S2) * Z + alpha0 * np.outer(M1, M1 @ Omega)"),
    ("rotation without the old basis", "return W_new.T @ (pinv_transpose(W_old) @ Phi)", "return W_new.T @ (W_old @ Phi)"),
    ("correlation not centred", "a = mu_true[i] - mu_true[i].mean()", "a = mu_true[i]"),
    ("matching minimises", "r, c = linear_sum_assignment(-Cm)", "r, c = linear_sum_assignment(Cm)"),
    ("batched keeps the highest loss", "best = int(ok[np.argmin(means[ok])])", "best = int(ok[np.argmax(means[ok])])"),
    ("VI without digamma", "p = rows * np.exp(scipy.special.digamma(gamma))[None, :]", "p = rows * gamma[None, :]"),
    ("VI drops the prior", "return phi, alpha + f @ phi", "return phi, f @ phi"),
    ("bound entropy sign", "h_z = -(f[:, None] * phi * logphi).sum()", "h_z = (f[:, None] * phi * logphi).sum()"),
    ("S2 with repeated tokens", "S2=int(np.sum(L * (L - 1)))", "S2=int(np.sum(L * L))"),
]
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_online.py", "tests/test_oracle_batched.py",
             "tests/test_oracle_vi.py"]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "tlda_oracle.py")).read()
    assert old in src, f"mutation site for {name!r} not found"
    (tmp_path / "oracle").mkdir()
    (tmp_path / "oracle" / "__init__.py").write_text("")
    (tmp_path / "oracle" / "tlda_oracle.py").write_text(src.replace(old, new, 1))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
    env = dict(os.environ, PYTHONPATH=f"{tmp_path}{os.pathsep}{ROOT}")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *PIN_FILES],
                       cwd=tmp_path, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name!r} passed every pin:\n{r.stdout[-800:]}"
