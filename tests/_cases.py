"""Shared seeded cases for the GPU tests: one event feeds both the FP64
oracle and the CUDA library (each runs its own start-up from the raw node
overlaps)."""
import functools

import numpy as np

from workload import standin
from workload.standin import make_event, make_queries, spec_for


@functools.lru_cache(maxsize=None)
def event(name, **over):
    return make_event(spec_for(name, **over))


def _key(over):
    return tuple(sorted(over.items()))


@functools.lru_cache(maxsize=None)
def _oracle(name, okey):
    import oracle
    return oracle.Model.from_event(event(name, **dict(okey)))


def oracle_model(name, **over):
    return _oracle(name, _key(over))


@functools.lru_cache(maxsize=None)
def _gpu(name, okey, form):
    import paper_2508_04172_gb300 as mf
    ev = event(name, **dict(okey))
    s = ev.spec
    return mf.Interpolant.from_overlaps(
        ev.nodes, standin.node_overlaps(ev), standin.standin_sigma(ev, ev.nodes), s.rank, s.eps,
        s.modes, ev.det, s.t0, s.dt, s.d_ref, ev.metric, ev.centre, s.tail_degree, form, sky=ev.sky,
        kernel=s.kernel)


def gpu_model(name, form="fp32", **over):
    return _gpu(name, _key(over), form)


def queries(name, Q, seed=None, **over):
    return make_queries(event(name, **over), Q, seed=seed)
