"""GB300-native staggered-fermion hot path (arXiv:1801.01473): the even/odd
staggered Dirac operator D_eo / D_oe, the multi-shift CG solve of
(m^2 - D_eo D_oe + sigma_i) x_i = b, the fermion force and the stout smearing of the
links with its force chain rule, as hand-written
CUDA kernels for sm_103a behind the C ABI of include/stg.h (libstg.so).

This package is the thin Python binding over that library; torch provides
device memory and streams.  Build the library with
``python -m paper_1801_01473_gb300.build``.
"""
from .api import (Gauge, Lattice, complex_convert, dslash, dslash_eo, dslash_host, dslash_eo_, dslash_multi_, dslash_oe, dslash_oe_, fermion_force,
                  gauge_action, gauge_force, md_kinetic, md_momenta, md_update_links_,
                  md_update_momenta_, mscg, rational_apply, mscg_batched, normal_op, normal_op_, normal_op_noalloc_, pack,
                  pseudofermion_action_value, stout_force, stout_smear, unpack)
from .autograd import PseudofermionAction, StoutSmear, pseudofermion_action, stout_smear_links
from . import md, rational
from .lib import StgError, lib

__all__ = ["Lattice", "Gauge", "complex_convert", "dslash", "dslash_host", "pack", "unpack", "dslash_eo", "dslash_oe", "dslash_eo_", "dslash_oe_",
           "dslash_multi_", "normal_op", "normal_op_", "normal_op_noalloc_", "mscg", "mscg_batched", "rational_apply",
           "pseudofermion_action_value", "fermion_force",
           "stout_smear", "stout_force", "gauge_action", "gauge_force", "md_momenta", "md_update_links_",
           "md_update_momenta_", "md_kinetic", "md", "PseudofermionAction", "pseudofermion_action", "StoutSmear",
           "stout_smear_links", "StgError", "lib"]
