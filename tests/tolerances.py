"""Tolerances that depart from the default rule, each demonstrated to be forced by FP32 arithmetic
in tests/test_fp32_bounds.py (the FP64 oracle run on inputs carrying FP32-sized errors).

The default rule (reading 17): a gradient tensor g matches the oracle's g_ref when
max|g - g_ref| <= 1e-3 max|g_ref| and, per element, |g - g_ref| <= 1e-3 (|g_ref| + floor max|g_ref|)
with floor = 1e-3; forward planes match within 1e-5 absolute."""

# Depth-gradient normal (K8) on FP32 planes that both sides share: one rounding of the
# alpha-normalised depth z = D / alpha moves the normal by up to ~3e-5 and the depth and alpha
# gradients beyond the default per-element floor.
NORMAL_FWD_TOL = 5e-5
NORMAL_GRAD_FLOOR = 1e-2

# Chains through the rasterizer (render -> depth_normal -> loss, render -> shade -> loss): the GPU
# chain works on FP32 rasterized planes, whose errors (up to ~4e-7 against the oracle's) the
# normal and the sun-visibility test amplify.
CHAIN_GRAD_FLOOR = 1e-2

# Size of the absolute errors of the FP32 rasterized planes that the demonstrations inject:
# half the largest forward error measured against the oracle.
FP32_PLANE_ERROR = 2e-7
