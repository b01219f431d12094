"""Mutation test of the oracle's pins.

Each mutant below plants one plausible mistake in a copy of ``oracle/`` -- a
dropped term or factor, a wrong sign, a wrong index, a transposed operand, a
wrong constant -- and runs the oracle's pin tests (``tests/test_oracle_*.py``
with their golden files) against that copy in a subprocess.  Every mutant must
make at least one pin fail; an unmutated copy must pass.  The mistakes are
planted in the CPU oracle only.

A mutant names the file, one source fragment that occurs exactly once in it,
and its replacement.  When the oracle's source changes, a fragment that no
longer occurs fails the test loudly rather than passing silently.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file under oracle/, fragment, replacement)
MUTANTS = [
    # B-splines (Definition 2.1)
    ("knots_drop_end", "bspline.py", "+ [1.0] * (p + 1))", "+ [1.0] * p)"),
    ("basis_den1_index", "bspline.py", "den1 = kn[l + d] - kn[l]", "den1 = kn[l + d + 1] - kn[l]"),
    ("basis_second_quotient", "bspline.py", "t += (kn[l + d + 1] - x) / den2", "t += (kn[l + d] - x) / den2"),
    ("basis_right_end", "bspline.py", "inside |= x == kn[l + 1]", "pass"),
    ("deriv_sign", "bspline.py", "D[:, l] -= p / den2", "D[:, l] += p / den2"),
    ("deriv_factor", "bspline.py", "D[:, l] += p / den1", "D[:, l] += 1.0 / den1"),
    ("periodic_shift_sign", "bspline.py", "out[:, i] = cardinal(p, np.mod(n_el * x - i, n_el))",
     "out[:, i] = cardinal(p, np.mod(n_el * x + i, n_el))"),
    ("periodic_chain_rule", "bspline.py", "out[:, i] = n_el * cardinal_deriv(",
     "out[:, i] = cardinal_deriv("),
    ("gauss_weights", "bspline.py", "return (g + 1.0) / 2.0, w / 2.0", "return (g + 1.0) / 2.0, w"),
    ("periodic_element_dofs", "bspline.py", "i = (e - p + a) % n_el", "i = (e + a) % n_el"),
    # geometry and metric (Secs. 2.2, 3.2)
    ("sphere_du_sign", "geometry.py", "Fu = cu / nrm - c", "Fu = cu / nrm + c"),
    ("sphere_dv_power", "geometry.py", "Fv = cv / nrm - c * (c @ cv)[..., None] / nrm**3",
     "Fv = cv / nrm - c * (c @ cv)[..., None] / nrm**2"),
    ("torus_dv_component", "geometry.py", "2 * np.pi * r * np.cos(tv)]", "2 * np.pi * r * np.sin(tv)]"),
    ("torus_du_radius", "geometry.py", "-2 * np.pi * rho * np.sin(tu)", "-2 * np.pi * r * np.sin(tu)"),
    ("metric_det_sign", "geometry.py", "det = K11 * K22 - K12 * K12", "det = K11 * K22 + K12 * K12"),
    ("metric_inverse_transposed", "geometry.py", "return a, K22 / a, -K12 / a, K11 / a",
     "return a, K11 / a, -K12 / a, K22 / a"),
    ("metric_offdiag_sign", "geometry.py", "return a, K22 / a, -K12 / a, K11 / a",
     "return a, K22 / a, K12 / a, K11 / a"),
    ("cube_face_sign", "geometry.py", "(1, 0, 2, -1.0),", "(1, 0, 2, +1.0),"),
    ("torus_area", "geometry.py", "return 4.0 * np.pi**2 * self.R * self.r", "return 2.0 * np.pi**2 * self.R * self.r"),
    # quadrature and assembly (Sec. 3.2)
    ("quad_element_size", "assembly.py", "/ (surf.n_u * surf.n_v) + 0 * U", "/ surf.n_u + 0 * U"),
    ("quad_point_index", "assembly.py", "U = ((eu[None, :, None, None] + g[None, None, None, :])",
     "U = ((eu[None, :, None, None] + g[None, None, :, None])"),
    ("local_index_transposed", "assembly.py", 'phi = np.einsum("yag,xbh->yxabgh", vv, vu)',
     'phi = np.einsum("yag,xbh->yxbagh", vv, vu)'),
    ("stiffness_cross_sign", "assembly.py", "gu = G11[:, :, None] * du + G12", "gu = G11[:, :, None] * du - G12"),
    ("mass_drop_measure", "assembly.py", "phi, W * a, phi))", "phi, W, phi))"),
    ("stiffness_drop_v_term", "assembly.py",
     'Se.append(np.einsum("yxkgh,yxgh,yxlgh->yxkl", du, W, gu)\n'
     '                  + np.einsum("yxkgh,yxgh,yxlgh->yxkl", dv, W, gv))',
     'Se.append(np.einsum("yxkgh,yxgh,yxlgh->yxkl", du, W, gu))'),
    ("assembly_cols", "assembly.py", "cols = np.tile(c, (1, nk)).ravel()", "cols = np.repeat(c, nk, axis=1).ravel()"),
    ("load_drop_measure", "assembly.py", 'fq = f(X) * quad["W"] * quad["a"][m]', 'fq = f(X) * quad["W"]'),
    ("evaluate_transposed", "assembly.py", '"ni,ji,nj->n", Bu, C, Bv', '"ni,ij,nj->n", Bu, C, Bv'),
    ("load_points_of_patch_zero", "assembly.py", 'X, _, _ = surf.map(m, quad["u"], quad["v"])',
     'X, _, _ = surf.map(0, quad["u"], quad["v"])'),
    ("load_local_index", "assembly.py", 'loc = np.einsum("yxkgh,yxgh->yxk", phi, fq)',
     'loc = np.einsum("yxkgh,yxhg->yxk", phi, fq)'),
    # glued space (Sec. 2.3)
    ("greville_window", "space.py", "kn[i + 1:i + p + 1].mean()", "kn[i:i + p].mean()"),
    ("no_gluing", "space.py", "first[j] = min(first[j], first[i])", "pass"),
    ("periodic_conn_shift", "space.py", "iv = (ev - p + kv) % s.n_v", "iv = (ev + kv) % s.n_v"),
    # white noise (Sec. 3.3)
    ("noise_no_sqrt", "noise.py", 'wq = np.sqrt(quad["W"] * quad["a"][m]) * xi[m]', 'wq = quad["W"] * quad["a"][m] * xi[m]'),
    ("noise_same_sample", "noise.py", "normals(seed, s, q, STREAM_NOISE)", "normals(seed, 0, q, STREAM_NOISE)"),
    ("noise_local_index", "noise.py", 'loc = np.einsum("yxkgh,yxgh->yxk", phi, wq)',
     'loc = np.einsum("yxkgh,yxhg->yxk", phi, wq)'),
    ("noise_adjoint_no_sqrt", "noise.py", 'out.append((np.sqrt(quad["W"] * quad["a"][m]) * val).ravel())',
     'out.append((quad["W"] * quad["a"][m] * val).ravel())'),
    ("noise_adjoint_point_index", "noise.py", 'val = np.einsum("yxkgh,yxk->yxgh", phi, gl)',
     'val = np.einsum("yxkgh,yxk->yxhg", phi, gl)'),
    ("philox_multiplier", "philox.py", "_M0 = np.uint64(0xD2511F53)", "_M0 = np.uint64(0xD2511F35)"),
    ("philox_weyl", "philox.py", "k1 = (k1 + _W1) & _MASK", "k1 = (k1 + _W0) & _MASK"),
    ("philox_round_words", "philox.py", "c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]",
     "c = [hi0 ^ c[1] ^ k0, lo1, hi1 ^ c[3] ^ k1, lo0]"),
    ("uniform_closed_at_zero", "philox.py", "+ b + np.uint64(1))", "+ b)"),
    ("box_muller_same_half", "philox.py", "z1 = rad * np.sin(2.0 * np.pi * u2)", "z1 = rad * np.cos(2.0 * np.pi * u2)"),
    ("box_muller_radius", "philox.py", "rad = np.sqrt(-2.0 * np.log(u1))", "rad = np.sqrt(-np.log(u1))"),
    # integer split, sinc sum, improved split, adjoint (Sec. 3.4)
    ("split_threshold", "fractional.py", "if bp < 1.0 / 3.0 and n >= 1:", "if bp < 2.0 / 3.0 and n >= 1:"),
    ("split_improved_value", "fractional.py", "return n - 1, (bp + 1.0) / 2.0, 2", "return n - 1, (bp + 1.0) / 3.0, 2"),
    ("sinc_weight_exponent", "fractional.py", "k * np.exp((1.0 - beta_frac) * y)", "k * np.exp(-beta_frac * y)"),
    ("sinc_weight_pi", "fractional.py", "c = math.sin(math.pi * beta_frac) / math.pi * k",
     "c = math.sin(math.pi * beta_frac) * k"),
    ("sinc_node_sign", "fractional.py", "y = l * k", "y = -l * k"),
    ("auto_step", "fractional.py", "k = math.pi ** 2 / math.log(3.0 * m / tol)", "k = 2.0 * math.pi ** 2 / math.log(3.0 * m / tol)"),
    ("auto_upper_tail", "fractional.py", "y_hi = math.log(3.0 * s / (g * tol)) / g",
     "y_hi = math.log(3.0 * s / (g * tol)) / (1.0 - g)"),
    ("auto_lower_tail", "fractional.py", "y_lo = math.log(tol * (1.0 - g) * mu / (3.0 * s)) / (1.0 - g)",
     "y_lo = math.log(tol * (1.0 - g) * mu / (3.0 * s)) / g"),
    ("scalar_sinc_step", "fractional.py", "sinc_rule(beta_frac, 2.0 / math.sqrt(K), -K, K)",
     "sinc_rule(beta_frac, 1.0 / math.sqrt(K), -K, K)"),
    ("shifted_operands_swapped", "fractional.py", "spla.splu((self.S + sigma * self.M).tocsc(), permc_spec",
     "spla.splu((self.M + sigma * self.S).tocsc(), permc_spec"),
    ("apply_drop_mass", "fractional.py", "    rhs = M @ v\n", "    rhs = v\n"),
    ("apply_shift_kappa", "fractional.py", "x = sh.solve(math.exp(yl) + kappa**2, rhs)", "x = sh.solve(math.exp(yl) + kappa, rhs)"),
    ("integer_extra_solve", "fractional.py", "        for _ in range(n - 1):\n            w = sh.solve(kappa**2, M @ w)\n        v = w",
     "        for _ in range(n):\n            w = sh.solve(kappa**2, M @ w)\n        v = w"),
    ("integer_drop_mass", "fractional.py", "            w = sh.solve(kappa**2, M @ w)\n        v = w",
     "            w = sh.solve(kappa**2, w)\n        v = w"),
    ("first_pass_extra_mass", "fractional.py", "u += cl * sh.solve(math.exp(yl) + kappa**2, w)",
     "u += cl * sh.solve(math.exp(yl) + kappa**2, M @ w)"),
    ("loss_drop_mass", "fractional.py", "L = float(np.sum(d * (M @ d)))", "L = float(np.sum(d * d))"),
    ("adjoint_rhs_drop_mass", "fractional.py", "gt = 2.0 * (M @ d)", "gt = 2.0 * d"),
    ("adjoint_kappa_sign", "fractional.py", "dk += -2.0 * kappa * cl * float(", "dk += 2.0 * kappa * cl * float("),
    # NURBS geometry maps (Sec. 2.2)
    ("nurbs_quotient_sign", "nurbs.py", "Fu = (Au - F * Wu) / W", "Fu = (Au + F * Wu) / W"),
    ("nurbs_drop_weight", "nurbs.py", "wP = cpw[..., :3] * w[..., None]", "wP = cpw[..., :3]"),
    ("nurbs_v_basis_for_u", "nurbs.py", 'Av = np.einsum("ni,nj,jic->nc", Nu, dNv, wP)',
     'Av = np.einsum("ni,nj,jic->nc", dNu, Nv, wP)'),
    ("nurbs_transposed_net", "nurbs.py", 'A = np.einsum("ni,nj,jic->nc", Nu, Nv, wP)',
     'A = np.einsum("ni,nj,ijc->nc", Nu, Nv, wP)'),
    ("nurbs_drop_weight_derivative", "nurbs.py", "Fv = (Av - F * Wv) / W", "Fv = Av / W"),
    # sqrt(M) by the Hale–Higham–Trefethen sum (Sec. 3.3)
    ("hht_midpoint", "sqrt_mass.py", "(np.arange(1, n_nodes + 1) - 0.5)", "(np.arange(1, n_nodes + 1) - 0.25)"),
    ("hht_prefactor", "sqrt_mass.py", "c = 2.0 * K * math.sqrt(lo)", "c = K * math.sqrt(lo)"),
    ("hht_jacobian_power", "sqrt_mass.py", "* dn / cn ** 2", "* dn / cn"),
    ("hht_shift_scale", "sqrt_mass.py", "w2 = lo * (sn / cn) ** 2", "w2 = math.sqrt(lo) * (sn / cn) ** 2"),
    ("hht_drop_outer_factor", "sqrt_mass.py", "    return A @ acc", "    return acc"),
    ("hht_parameter", "sqrt_mass.py", "q = 1.0 - lo / hi", "q = lo / hi"),
    ("hht_no_reflection", "sqrt_mass.py", "far = t > 0.5 * K", "far = t > K"),
    ("hht_reflection_parameter", "sqrt_mass.py", "w2[far] = lo / kp2 * (cnu / snu) ** 2",
     "w2[far] = hi * (cnu / snu) ** 2"),
    ("bounds_diagonal_only", "sqrt_mass.py", "hi = float(np.abs(M).sum(axis=1).max())", "hi = float(M.diagonal().max())"),
    ("bounds_diagonal_max", "sqrt_mass.py", "return lam * float(M.diagonal().min()), hi",
     "return lam * float(M.diagonal().max()), hi"),
    ("bounds_unscaled", "sqrt_mass.py", "A / d[:, :, None] / d[:, None, :]", "A / d[:, :, None]"),
    ("adjoint_drop_integer_term", "fractional.py", "dk += -2.0 * kappa * float(np.sum(lam * (M @ ws[i])))",
     "pass"),
    ("adjoint_pass_drop_mass", "fractional.py", "            dout = M @ dLdr  # r = M v_prev",
     "            dout = dLdr  # r = M v_prev"),
    ("adjoint_pass_wrong_iterates", "fractional.py", "for cl, x, z in zip(c, xss[p_], zs):",
     "for cl, x, z in zip(c, xss[0], zs):"),
]

CONFTEST = (
    "import os, sys\n"
    "sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))\n"
    "def pytest_configure(config):\n"
    "    config.addinivalue_line('markers', 'gpu: needs a CUDA GPU')\n"
)


def _pin_files():
    return sorted(f for f in os.listdir(os.path.join(ROOT, "tests"))
                  if f.startswith("test_oracle_") and f.endswith(".py") and f != os.path.basename(__file__))


def _copy_tree(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    td = os.path.join(dst, "tests")
    os.makedirs(td)
    for f in _pin_files():
        shutil.copy(os.path.join(ROOT, "tests", f), td)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(td, "golden"))
    shutil.copy(os.path.join(ROOT, "wm_workloads.py"), dst)   # seeded inputs and geometry nets
    with open(os.path.join(td, "conftest.py"), "w") as fh:
        fh.write(CONFTEST)


def _mutate(dst, fname, old, new):
    path = os.path.join(dst, "oracle", fname)
    with open(path) as fh:
        src = fh.read()
    count = src.count(old)
    if count != 1:
        raise AssertionError(f"fragment occurs {count} times in oracle/{fname}: {old!r}")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))


# pin files that exercise a module most directly run first (pytest -x stops at
# the first failure); every pin file runs if those pass
FIRST = {"bspline.py": ["test_oracle_bspline.py"], "geometry.py": ["test_oracle_geometry.py"],
         "assembly.py": ["test_oracle_assembly.py"], "space.py": ["test_oracle_assembly.py"],
         "noise.py": ["test_oracle_noise.py"], "philox.py": ["test_oracle_noise.py"],
         "fractional.py": ["test_oracle_sinc.py", "test_oracle_fractional.py"],
         "sqrt_mass.py": ["test_oracle_sqrt_mass.py"], "nurbs.py": ["test_oracle_nurbs.py"]}


def _run_pins(dst, fname=None):
    env = dict(os.environ, PYTHONPATH=dst, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1",
               OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    first = FIRST.get(fname, [])
    files = first + [f for f in _pin_files() if f not in first]
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += [os.path.join(dst, "tests", f) for f in files]
    res = subprocess.run(cmd, cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return res.returncode, res.stdout[-2000:]


def _case(tmp, idx, mutant):
    dst = os.path.join(tmp, f"m{idx:02d}")
    _copy_tree(dst)
    fname = None
    if mutant is not None:
        _, fname, old, new = mutant
        _mutate(dst, fname, old, new)
    return _run_pins(dst, fname)


def test_mutant_fragments_are_unique():
    pins = set(_pin_files())
    assert set(FIRST) == {m[1] for m in MUTANTS} and all(set(v) <= pins for v in FIRST.values())
    for name, fname, old, new in MUTANTS:
        with open(os.path.join(ROOT, "oracle", fname)) as fh:
            assert fh.read().count(old) == 1, (name, old)
        assert old != new, name
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)


def test_every_mutant_fails_a_pin(tmp_path):
    jobs = [None] + MUTANTS
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = [ex.submit(_case, str(tmp_path), i, m) for i, m in enumerate(jobs)]
        results = [f.result() for f in futs]
    rc0, out0 = results[0]
    assert rc0 == 0, "unmutated oracle copy fails its pins:\n" + out0
    survivors, broken = [], []
    for m, (rc, out) in zip(MUTANTS, results[1:]):
        if rc == 0:
            survivors.append(m[0])
        elif rc != 1:  # collection error, usage error: the mutant did not run as a plausible mistake
            broken.append((m[0], rc, out))
    assert not broken, broken
    assert not survivors, f"mutants no pin detects: {survivors}"
