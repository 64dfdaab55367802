"""Seeded synthetic workloads for the meshfree log-likelihood path.

This package only draws random inputs and evaluates the closed-form stand-in
overlap model that replaces waveform-generation + data (the paper computes the
node overlaps z and cross terms sigma from IMRPhenomXHM and detector strain,
Sec. II C 2; neither exists here).  It holds none of the method's own
arithmetic: no SVD, no RBF fit, no spline, no spherical harmonics and no
log-likelihood.  Both the FP64 oracle and the GPU library consume its output.
"""
from .standin import (CONFIGS, Spec, spec_for, make_event, make_queries,
                      standin_z, standin_sigma, ball, eps_rule)

__all__ = ["CONFIGS", "Spec", "spec_for", "make_event", "make_queries",
           "standin_z", "standin_sigma", "ball", "eps_rule"]
