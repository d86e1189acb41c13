"""Seeded synthetic inputs for the CT augmentation workloads.

This package only *draws* inputs: CT-like phantoms with their label maps,
random affine transforms, photometric/noise parameters, probability maps and
upstream gradients.  It contains none of the augmentation arithmetic (no
warping, interpolation, noise generation or loss), so that both the FP64
oracle and the CUDA library can consume the very same inputs without sharing
any computation.

The paper's own data (130 labelled CT scans, Sec. 6.A) is not available; the
phantoms below stand in for it with the structure described in Sec. 4/5.A:
air at -1000 HU, an ellipsoidal body with Gaussian texture, soft-tissue
"organs" with labels 1..4 and bone blobs with label 5.
"""
from .phantom import make_phantom, PhantomSpec
from .params import random_affine, random_photometric, AffineSpec
from . import workloads

__all__ = [
    "make_phantom",
    "PhantomSpec",
    "random_affine",
    "random_photometric",
    "AffineSpec",
    "workloads",
]
