"""Error norms shared by the GPU parity tests.

Fields: ||a - r||_2 / ||r||_2 over the whole field.  Correlators: per
(channel, momentum), ||C(.) - C_ref(.)||_2 / ||C_ref(.)||_2 over t; a
(channel, momentum) whose reference norm is below 1e-12 of the largest one
is measured against that largest norm instead (it is zero up to rounding).
"""
import numpy as np

# FP32 arithmetic on FP32-representable inputs; BF16 storage.
TOL_F32 = 1e-5
TOL_BF16 = 2e-2


def field_err(a, ref) -> float:
    a = np.asarray(a)
    ref = np.asarray(ref)
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))


def field_err_t(a, ref, t_axis: int = 0) -> float:
    """Largest per-timeslice relative error: max over t of ||a_t - r_t|| / ||r_t||.

    A smeared field's magnitude varies by orders of magnitude between
    timeslices (the source envelope), so an error confined to the small
    timeslices hardly moves the global norm; this one sees it."""
    a = np.moveaxis(np.asarray(a), t_axis, 0)
    ref = np.moveaxis(np.asarray(ref), t_axis, 0)
    d = np.linalg.norm((a - ref).reshape(a.shape[0], -1), axis=1)
    n = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    # a timeslice the reference leaves at zero (a point source's other timeslices)
    # is measured against the largest timeslice norm
    n = np.where(n > 1e-12 * n.max(), n, n.max())
    return float((d / n).max())


def corr_err(C, C_ref) -> float:
    C = np.asarray(C)
    C_ref = np.asarray(C_ref)
    diff = np.linalg.norm(C - C_ref, axis=-1)
    norm = np.linalg.norm(C_ref, axis=-1)
    floor = 1e-12 * norm.max()
    denom = np.where(norm > floor, norm, norm.max())
    return float((diff / denom).max())


def to_bf16_complex(a: np.ndarray) -> np.ndarray:
    """Round real and imaginary parts to bfloat16 (RNE) with torch on the CPU."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    re = t.real.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    im = t.imag.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    return torch.complex(re, im).numpy()


def proj_err(C, C_ref, abs_scale) -> float:
    """Error of momentum-projected correlators C[..., p, t] measured against
    the scale of the sum that produced them: per (channel, momentum),
    ||C - C_ref||_2 over t divided by ||A||_2 over t, where A(t) =
    sum_x |c(x)| is the sum of the site values' magnitudes (the same for
    every momentum).  At p != 0 a smooth field's correlator is a heavily
    cancelling sum, and FP32 site values bound the accuracy of any such sum
    relative to A, not to the (much smaller) result."""
    C = np.asarray(C)
    C_ref = np.asarray(C_ref)
    A = np.asarray(abs_scale)
    diff = np.linalg.norm(C - C_ref, axis=-1)
    return float((diff / np.linalg.norm(A, axis=-1)[..., None]).max())
