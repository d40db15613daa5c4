"""The pins must be sharp: each plausible mistake planted in a copy of the
oracle source (on the CPU, in a temporary build) must fail at least one pin.
The real oracle source is never modified."""
import os

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "trid_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("thomas_forward_sign", "ds[i] = r * (d[i] - a[i] * ds[i - 1]);",
     "ds[i] = r * (d[i] + a[i] * ds[i - 1]);"),
    ("thomas_backward_sign", "x[i] = ds[i] - cs[i] * x[i + 1];", "x[i] = ds[i] + cs[i] * x[i + 1];"),
    ("thomas_pivot_index", "double den = b[i] - a[i] * cs[i - 1];",
     "double den = b[i] - a[i] * cs[i > 1 ? i - 2 : 0];"),
    ("pcr_transposed_operand", "am = A0[i - s]; cm = C0[i - s];", "am = C0[i - s]; cm = A0[i - s];"),
    ("pcr_sign", "double den = 1.0 - A0[i] * cm - C0[i] * ap;",
     "double den = 1.0 - A0[i] * cm + C0[i] * ap;"),
    ("pcr_rounds", "while (((int64_t)1 << P) < n) ++P;", "while (((int64_t)2 << P) < n) ++P;"),
    ("tiled_dropped_term", "ah[i] = ah[i] - ch[i] * ah[i + 1];", "ah[i] = ah[i];"),
    ("tiled_reduced_diag", "rb[2 * k] = 1.0 - ch[s] * ah[s + 1];", "rb[2 * k] = 1.0;"),
    ("lines_row_offset", "int rc = orc_thomas(n, a + k * n, b + k * n, c + k * n, d + k * n, x + k * n);",
     "int rc = orc_thomas(n, a + k, b + k * n, c + k * n, d + k * n, x + k * n);"),
    ("lines_row_length", "int rc = orc_thomas(n, a + k * n, b + k * n, c + k * n, d + k * n, x + k * n);",
     "int rc = orc_thomas(n - 1, a + k * n, b + k * n, c + k * n, d + k * n, x + k * n);"),
    ("lines_row_count", "for (int64_t k = 0; k < nsys; ++k) {\n        int rc = orc_thomas(n,",
     "for (int64_t k = 0; k + 1 < nsys; ++k) {\n        int rc = orc_thomas(n,"),
    ("f32_forward_sign", "dp[i] = r * (d[i] - a[i] * dp[i - 1]);",
     "dp[i] = r * (d[i] + a[i] * dp[i - 1]);"),
    ("f32_line_stride", "for (int64_t i = 0; i < n; ++i) out[base + i * st] = lx[i];",
     "for (int64_t i = 0; i < n; ++i) out[base + i] = lx[i];"),
    ("mesh_accumulate", "if (accumulate) out[p] += lx[i]; else out[p] = lx[i];", "out[p] = lx[i];"),
    ("adi_stencil_centre", "dd[p] = lambda * (s - 2.0 * ndim * u[p]);", "dd[p] = lambda * (s - ndim * u[p]);"),
    ("adi_operator_diag", "lb[i] = bnd ? 1.0 : 1.0 + 2.0 * lambda;", "lb[i] = bnd ? 1.0 : 1.0 + lambda;"),
    ("adi_missing_z", "if (ndim == 3) s += u[p - stride[2]] + u[p + stride[2]];",
     "if (ndim == 4) s += u[p - stride[2]] + u[p + stride[2]];"),
    ("adjoint_not_transposed", "ta[i] = (i == 0) ? 0.0 : c[i - 1];", "ta[i] = (i == 0) ? 0.0 : a[i];"),
    ("adjoint_wrong_neighbour", "gc[i] = (i == n - 1) ? 0.0 : -gd[i] * x[i + 1];",
     "gc[i] = (i == n - 1) ? 0.0 : -gd[i] * x[i];"),
    ("dense_no_pivoting", "if (v > best) { best = v; piv = r; }", "if (0) { best = v; piv = r; }"),
    ("adi2v_face_mean", "double kr = 0.5 * (kappa[p] + kappa[p + 1]);",
     "double kr = 0.5 * (kappa[p] + kappa[p]);"),
    ("adi2v_rhs_sign", "d[p] = -cx[p] * (u[p + 1] - u[p]) + ax[p] * (u[p] - u[p - 1])",
     "d[p] = -cx[p] * (u[p + 1] - u[p]) - ax[p] * (u[p] - u[p - 1])"),
    ("adi2v_grad_transposed_stencil", "gu[p + 1] += -co[2][p] * gm;", "gu[p + 1] += -co[0][p] * gm;"),
    ("adi2v_grad_dropped_stencil_term", "G[0][p] += gm * (u[p] - u[p - 1]);", "G[0][p] += 0.0;"),
    ("adi2v_grad_face", "gkx[p] += lam * (G[1][p] - G[2][p]);", "gkx[p] += lam * (G[1][p] - G[0][p]);"),
    ("adi2v_grad_loss_scale", "g[p] = 2.0 * r / (double)n;", "g[p] = r / (double)n;"),
    ("adi2v_grad_wrong_state", "const double *u = U + tt * n, *w = W + tt * n",
     "const double *u = U + (tt + 1) * n, *w = W + tt * n"),
]


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, orig, bad):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for {name} not unique/present"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(orig, bad))
    so = str(tmp_path / "libmutant.so")
    import subprocess
    subprocess.run(["gcc", *oracle.CFLAGS, str(src), "-o", so, "-lm"], check=True)
    lib = oracle.load(so)
    failed = []
    for pin in pins.ALL_PINS:
        try:
            ok, _ = pin(lib)
        except (ZeroDivisionError, ValueError, FloatingPointError, OverflowError,
                __import__("numpy").linalg.LinAlgError):
            ok = False
        if not ok:
            failed.append(pin.__name__)
    assert failed, f"planted mistake {name} passed every pin"
