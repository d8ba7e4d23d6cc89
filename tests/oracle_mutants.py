"""Plausible mistakes planted in the oracle, one at a time, on the CPU.

Loaded as a pytest plugin (``-p oracle_mutants``) by
``test_oracle_mutations.py`` in a child process; the environment variable
ORACLE_MUTANT names the mistake.  Each mistake is a text substitution in one
oracle source file: a Python module is re-executed from the altered text into
its own namespace (so every caller, the pins included, sees the altered
functions), and the C tracer is recompiled from the altered text into a
temporary directory and loaded in place of the real one.  The oracle's files
on disk are never changed.

The mistakes are the kinds the pins must catch: a dropped term, a wrong sign,
a wrong index or offset, a transposed operand, a wrong constant.
"""

import os
import tempfile

# name -> (pin file that must fail, oracle source file, [(old text, new text), ...])
MUTANTS = {
    # ---- tv.py: gradient, operator, CG ----
    "grad_periodic_boundary": ("test_oracle_tv.py", "tv.py", [
        ("    gx[:, :-1] = u[:, 1:] - u[:, :-1]\n",
         "    gx[:, :-1] = u[:, 1:] - u[:, :-1]\n    gx[:, -1] = u[:, 0] - u[:, -1]\n")]),
    "grad_adj_dropped_term": ("test_oracle_tv.py", "tv.py", [
        ("    out[:, :-1] -= wx[:, :-1]\n", "")]),
    "grad_adj_swapped_components": ("test_oracle_tv.py", "tv.py", [
        ("    out[:, 1:] += wx[:, :-1]\n    out[:, :-1] -= wx[:, :-1]\n"
         "    out[1:, :] += wy[:-1, :]\n    out[:-1, :] -= wy[:-1, :]\n",
         "    out[:, 1:] += wy[:, :-1]\n    out[:, :-1] -= wy[:, :-1]\n"
         "    out[1:, :] += wx[:-1, :]\n    out[:-1, :] -= wx[:-1, :]\n")]),
    "operator_grad_term_minus": ("test_oracle_tv.py", "tv.py", [
        ("y += c_grad * grad_adj(gx, gy).ravel()", "y -= c_grad * grad_adj(gx, gy).ravel()")]),
    "operator_drops_identity_term": ("test_oracle_tv.py", "tv.py", [
        ("            y += c_id * x\n", "            pass\n")]),
    "cg_beta_inverted": ("test_oracle_tv.py", "tv.py", [
        ("p = r + (rr_new / rr) * p", "p = r + (rr / rr_new) * p")]),
    "cg_residual_sign": ("test_oracle_tv.py", "tv.py", [
        ("r = r - a * q", "r = r + a * q")]),
    "cg_residual_ignores_warm_start": ("test_oracle_tv.py", "tv.py", [
        ("    r = rhs - op(u)\n", "    r = rhs.copy()\n")]),
    "cg_tolerance_on_squared_norm": ("test_oracle_tv.py", "tv.py", [
        ("np.sqrt(np.real(rr)) <= rel_tol * rhs_norm", "np.real(rr) <= rel_tol * rhs_norm")]),
    "cg_refresh_one_step_early": ("test_oracle_tv.py", "tv.py", [
        ("done % refresh_every == 0 and done < iters", "(done - 1) % refresh_every == 0 and done < iters")]),
    "cg_refresh_keeps_old_rr": ("test_oracle_tv.py", "tv.py", [
        ("            rr = r @ r\n", "")]),
    "cg_refresh_restarts_direction": ("test_oracle_tv.py", "tv.py", [
        ("            rr = r @ r\n", "            rr = r @ r\n            p = r.copy()\n")]),
    "sb_refresh_matrix_ignored": ("test_oracle_tv.py", "tv.py", [
        ("refresh_op=op_refresh)", "refresh_op=None)")]),
    # ---- tv.py: split Bregman ----
    "shrink_half_threshold": ("test_oracle_tv.py", "tv.py", [
        ("np.abs(xr) > gamma, x - gamma * np.sign(xr)",
         "np.abs(xr) > 0.5 * gamma, x - 0.5 * gamma * np.sign(xr)")]),
    "shrink_unsigned": ("test_oracle_tv.py", "tv.py", [
        ("x - gamma * np.sign(xr)", "x - gamma")]),
    "sb_v_is_d_plus_b": ("test_oracle_tv.py", "tv.py", [
        ("grad_adj(dx - bx, dy - by)", "grad_adj(dx + bx, dy + by)")]),
    "sb_bregman_sign": ("test_oracle_tv.py", "tv.py", [
        ("bx = bx + gx - dx", "bx = bx - gx + dx")]),
    "sb_threshold_lambda": ("test_oracle_tv.py", "tv.py", [
        ("dx = shrink(gx + bx, 1.0 / lam)", "dx = shrink(gx + bx, lam)")]),
    "sb_shrink_drops_b": ("test_oracle_tv.py", "tv.py", [
        ("dy = shrink(gy + by, 1.0 / lam)", "dy = shrink(gy, 1.0 / lam)")]),
    "sb_data_term_unscaled": ("test_oracle_tv.py", "tv.py", [
        ("atf = alpha * (A.T @ f)", "atf = A.T @ f")]),
    "sb_inner_cg_not_warm_started": ("test_oracle_tv.py", "tv.py", [
        ("u, _ = cg(op, rhs, u_old, inner, rel_tol=cg_tol,", "u, _ = cg(op, rhs, np.zeros_like(u_old), inner, rel_tol=cg_tol,")]),
    "sb_update_size_l2": ("test_oracle_tv.py", "tv.py", [
        ("updates.append(float(np.abs(u - u_old).sum()))",
         "updates.append(float(np.sqrt(((u - u_old) ** 2).sum())))")]),
    "tv_objective_drops_half": ("test_oracle_tv.py", "tv.py", [
        ("return 0.5 * alpha * float(res @ res)", "return alpha * float(res @ res)")]),
    "stop_rule_against_previous_update": ("test_oracle_tv.py", "tv.py", [
        ("updates[-1] < stop_rel_update * updates[0]", "updates[-1] < stop_rel_update * updates[-2]")]),
    # ---- tv.py: resolvent, Chambolle-Pock ----
    "resolvent_rhs_drops_tau": ("test_oracle_tv.py", "tv.py", [
        ("rhs = u_tilde.ravel() + tau * alpha * (A.T @ g)", "rhs = u_tilde.ravel() + alpha * (A.T @ g)")]),
    "cp_primal_step_sign": ("test_oracle_tv.py", "tv.py", [
        ("ut = u - tau * grad_adj(px, py).ravel()", "ut = u + tau * grad_adj(px, py).ravel()")]),
    "cp_dual_ascent_sign": ("test_oracle_tv.py", "tv.py", [
        ("px = np.clip(px + sigma * gx, -1.0, 1.0)", "px = np.clip(px - sigma * gx, -1.0, 1.0)")]),
    "cp_extrapolates_from_old_iterate": ("test_oracle_tv.py", "tv.py", [
        ("ubar = u_new + theta * (u_new - u)", "ubar = u + theta * (u_new - u)")]),
    "cp_resolvent_not_warm_started": ("test_oracle_tv.py", "tv.py", [
        ("u_new, _ = resolvent(A, shape, tau, alpha, ut, g, inner, u0=u)",
         "u_new, _ = resolvent(A, shape, tau, alpha, ut, g, inner, u0=np.zeros_like(u))")]),
    # ---- tv.py: surrogate ----
    "point_response_off_centre": ("test_oracle_tv.py", "tv.py", [
        ("e[(n // 2) * n + n // 2] = 1.0", "e[(n // 2) * n + n // 2 - 1] = 1.0")]),
    "stencil_not_symmetrised": ("test_oracle_tv.py", "tv.py", [
        ("0.5 * (h[c + di, c + dj] + h[c - di, c - dj])", "h[c + di, c + dj]")]),
    "stencil_wrong_mirror_index": ("test_oracle_tv.py", "tv.py", [
        ("0.5 * (h[c + di, c + dj] + h[c - di, c - dj])", "0.5 * (h[c + di, c + dj] + h[c - di, c + dj])")]),
    "stencil_window_max_norm": ("test_oracle_tv.py", "tv.py", [
        ("if shape == \"disc\" and di * di + dj * dj > r * r:",
         "if shape == \"disc\" and max(abs(di), abs(dj)) > r:")]),
    "surrogate_periodic_wrap": ("test_oracle_tv.py", "tv.py", [
        ("ti, tj = (ii + di).ravel(), (jj + dj).ravel()",
         "ti, tj = (ii + di).ravel() % n, (jj + dj).ravel() % n")]),
    # ---- radon.py ----
    "bin_offsets_shifted": ("test_oracle_radon.py", "radon.py", [
        ("- 0.5 * (n_bins - 1)", "- 0.5 * n_bins")]),
    "clip_edge_full_length": ("test_oracle_radon.py", "radon.py", [
        ("factor = 0.5", "factor = 1.0")]),
    "quantize_scale_is_row_sum": ("test_oracle_radon.py", "radon.py", [
        ("np.maximum.reduceat(A.data", "np.add.reduceat(A.data")]),
    "dequantize_drops_scale": ("test_oracle_radon.py", "radon.py", [
        ("return sp.diags(s.astype(np.float64)) @ Qd", "return Qd")]),
    # ---- siddon.c ----
    "c_edge_full_length": ("test_oracle_radon.py", "siddon.c", [
        ("e[cnt].val = 0.5;", "e[cnt].val = 1.0;")]),
    "c_bin_offset_shifted": ("test_oracle_radon.py", "siddon.c", [
        ("(double)b - 0.5 * (double)(n_bins - 1)", "(double)b - 0.5 * (double)n_bins")]),
    "c_rows_bin_major": ("test_oracle_radon.py", "siddon.c", [
        ("row_nnz[(int64_t)kk * n_bins + b] = m;", "row_nnz[(int64_t)b * n_kept + kk] = m;"),
        ("const int64_t q = (int64_t)kk * n_bins + b;", "const int64_t q = (int64_t)b * n_kept + kk;")]),
    "c_pixel_index_transposed": ("test_oracle_radon.py", "siddon.c", [
        ("e[cnt].col = i * n + j;\n            e[cnt].val = len;",
         "e[cnt].col = j * n + i;\n            e[cnt].val = len;")]),
    "c_sin_sign": ("test_oracle_radon.py", "siddon.c", [
        ("*s = sin(th);", "*s = -sin(th);")]),
    "c_drops_short_segments": ("test_oracle_radon.py", "siddon.c", [
        ("#define ORACLE_MIN_LEN 1e-12", "#define ORACLE_MIN_LEN 1e-3")]),
    "c_grid_planes_shifted": ("test_oracle_radon.py", "siddon.c", [
        ("((double)m - 0.5 * n - x0) / dx", "((double)m - 0.5 * n + 0.5 - x0) / dx")]),
    "c_midpoint_lookup_off_by_one": ("test_oracle_radon.py", "siddon.c", [
        ("int j = (int)floor(x0 + tm * dx + half);", "int j = (int)floor(x0 + tm * dx + half + 0.5);")]),
    "c_planes_not_reversed": ("test_oracle_radon.py", "siddon.c", [
        ("    if (dx < 0) {\n        for (int a = 0, b = n; a < b; ++a, --b) {",
         "    if (dx > 0) {\n        for (int a = 0, b = n; a < b; ++a, --b) {")]),
    "c_boundary_rays_dropped": ("test_oracle_radon.py", "siddon.c", [
        ("if (v < -half || v > half) return 0;", "if (v <= -half || v >= half) return 0;")]),
    "c_angle_step_wrong": ("test_oracle_radon.py", "siddon.c", [
        ("double th = (double)k * ORACLE_PI / (double)n_total;", "double th = (double)k * ORACLE_PI / (double)(n_total - 1);")]),
    "c_keeps_wrong_angles": ("test_oracle_radon.py", "siddon.c", [
        ("oracle_direction(kk * keep_every, n_total, &c, &s);\n        for (int b = 0; b < n_bins; ++b) {\n            const double sb = (double)b - 0.5 * (double)(n_bins - 1);\n            const int m = trace_ray(n, c, s, sb, e, tx, ty);\n            row_nnz",
         "oracle_direction(kk, n_total, &c, &s);\n        for (int b = 0; b < n_bins; ++b) {\n            const double sb = (double)b - 0.5 * (double)(n_bins - 1);\n            const int m = trace_ray(n, c, s, sb, e, tx, ty);\n            row_nnz"),
        ("oracle_direction(kk * keep_every, n_total, &c, &s);\n        for (int b = 0; b < n_bins; ++b) {\n            const double sb = (double)b - 0.5 * (double)(n_bins - 1);\n            const int m = trace_ray(n, c, s, sb, e, tx, ty);\n            const int64_t q",
         "oracle_direction(kk, n_total, &c, &s);\n        for (int b = 0; b < n_bins; ++b) {\n            const double sb = (double)b - 0.5 * (double)(n_bins - 1);\n            const int m = trace_ray(n, c, s, sb, e, tx, ty);\n            const int64_t q")]),
    # ---- fourier.py ----
    "rho_centre_shifted": ("test_oracle_fourier.py", "fourier.py", [
        ("- (n_bins // 2)) / n_bins", "- (n_bins - 1) / 2.0) / n_bins")]),
    "pixel_centre_no_half": ("test_oracle_fourier.py", "fourier.py", [
        ("(jj - n / 2.0 + 0.5).ravel(), (ii - n / 2.0 + 0.5).ravel()",
         "(jj - n / 2.0).ravel(), (ii - n / 2.0).ravel()")]),
    "pixel_centre_axes_swapped": ("test_oracle_fourier.py", "fourier.py", [
        ("(jj - n / 2.0 + 0.5).ravel(), (ii - n / 2.0 + 0.5).ravel()",
         "(ii - n / 2.0 + 0.5).ravel(), (jj - n / 2.0 + 0.5).ravel()")]),
    "nudft_sign": ("test_oracle_fourier.py", "fourier.py", [
        ("np.exp(-1j * (np.outer(wx, x) + np.outer(wy, y)))", "np.exp(1j * (np.outer(wx, x) + np.outer(wy, y)))")]),
    "sinogram_dft_sign": ("test_oracle_fourier.py", "fourier.py", [
        ("phase = np.exp(-1j * np.outer(", "phase = np.exp(1j * np.outer(")]),
    "gaussian_exponent_sign": ("test_oracle_fourier.py", "fourier.py", [
        ("np.exp(-((w[:, None] - eta) ** 2) / (4.0 * tau))", "np.exp(((w[:, None] - eta) ** 2) / (4.0 * tau))")]),
    "gaussian_width_tau": ("test_oracle_fourier.py", "fourier.py", [
        ("np.exp(-((w[:, None] - eta) ** 2) / (4.0 * tau))", "np.exp(-((w[:, None] - eta) ** 2) / (2.0 * tau))")]),
    "deconvolution_sign": ("test_oracle_fourier.py", "fourier.py", [
        ("np.exp(k * k * tau)", "np.exp(-k * k * tau)")]),
    "half_pixel_phase_sign": ("test_oracle_fourier.py", "fourier.py", [
        ("np.exp(-0.5j * (self.wx + self.wy))", "np.exp(0.5j * (self.wx + self.wy))")]),
    "gridding_scale_one_factor": ("test_oracle_fourier.py", "fourier.py", [
        ("1.0 / (self.m_r * self.m_r * math.sqrt(self.n_bins))", "1.0 / (self.m_r * math.sqrt(self.n_bins))")]),
    "fused_matrix_transposed": ("test_oracle_fourier.py", "fourier.py", [
        ("(self.G.T @ self.G)", "(self.G @ self.G.T)")]),
    "fused_skips_ifft": ("test_oracle_fourier.py", "fourier.py", [
        ("P = np.fft.ifft2((C @ h).reshape(m_r, m_r)) * (m_r * m_r)", "P = (C @ h).reshape(m_r, m_r)")]),
    "fourier_point_response_unscaled": ("test_oracle_fourier.py", "fourier.py", [
        ("np.cos(wx * dj + wy * di).sum() / n_bins", "np.cos(wx * dj + wy * di).sum()")]),
    "default_tau_per_n": ("test_oracle_fourier.py", "fourier.py", [
        ("return m_sp / float(n * n)", "return m_sp / float(n)")]),
    "deconvolution_not_centred": ("test_oracle_fourier.py", "fourier.py", [
        ("k = np.arange(n, dtype=np.float64) - n // 2\n    return math.sqrt",
         "k = np.arange(n, dtype=np.float64)\n    return math.sqrt")]),
    "grid_placement_not_centred": ("test_oracle_fourier.py", "fourier.py", [
        ("k = (np.arange(n) - n // 2) % m_r", "k = np.arange(n) % m_r")]),
    "exact_normal_drops_conj": ("test_oracle_fourier.py", "fourier.py", [
        ("return np.real(self.F.conj().T @ (self.F @ mu))", "return np.real(self.F.T @ (self.F @ mu))")]),
    "exact_adjoint_drops_conj": ("test_oracle_fourier.py", "fourier.py", [
        ("return np.real(self.s.F.conj().T @ c)", "return np.real(self.s.F.T @ c)")]),
    "adjoint_drops_conj_phase": ("test_oracle_fourier.py", "fourier.py", [
        ("s = self.G.T @ (np.conj(self.phase) * np.asarray(c))", "s = self.G.T @ (self.phase * np.asarray(c))")]),
    "adjoint_keeps_imaginary_part": ("test_oracle_fourier.py", "fourier.py", [
        ("return np.real(self.scale() * self.crop(P)).ravel()", "return np.abs(self.scale() * self.crop(P)).ravel()")]),
}

_ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def _altered(path, subs):
    with open(path) as fh:
        src = fh.read()
    for old, new in subs:
        if src.count(old) < 1:
            raise RuntimeError("mutant text not found in %s: %r" % (path, old[:60]))
        src = src.replace(old, new)
    return src


def apply(name):
    """Plants mutant ``name`` in this process's oracle."""
    _, fname, subs = MUTANTS[name]
    path = os.path.join(_ORACLE, fname)
    src = _altered(path, subs)
    if fname.endswith(".c"):
        from oracle import _native

        out = tempfile.mkdtemp(prefix="oracle_mutant_")
        alt = os.path.join(out, "siddon.c")
        with open(alt, "w") as fh:
            fh.write(src)
        _native._SRC, _native._OUT_DIR = alt, out
        _native._LIB = os.path.join(out, "liboracle_siddon.so")
        _native._lib = None
        _native.lib()
    else:
        import importlib

        mod = importlib.import_module("oracle." + fname[:-3])
        exec(compile(src, path, "exec"), mod.__dict__)


def pytest_configure(config):
    name = os.environ.get("ORACLE_MUTANT", "")
    if name:
        apply(name)
        print("oracle mutant planted: %s" % name)
