"""Helpers shared by the GPU tests (no computation of the estimator here)."""
import numpy as np


def to_np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
