"""Shared test fixtures.  ``gpu`` marks tests that need a CUDA device (run with -m gpu)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built C-ABI library")


def oracle_problem(w, **overrides):
    """Oracle problem for a synthetic workload; the oracle computes its own grey constants and
    source deposit from the workload's spectrum and source list."""
    from oracle import closure as cl, model as md
    kind, par = w.spectrum
    grey = cl.grey_constants(kind, par, w.ns)
    src = cl.deposit_sources(w.nH.shape, w.dx, w.src_ijk, w.src_rate, grey["eps"])
    args = dict(nx=w.nx, ny=w.ny, nz=w.nz, dx=w.dx, ns=w.ns, nH=w.nH, src=src, grey=grey,
                y_he=w.y_he, bc=w.bc, theta=w.theta, u_e=w.u_e, u_n=w.u_n, u_E=w.u_E,
                model=w.model, kappa_total=w.kappa_total, kappa_planck=w.kappa_planck, mu=w.mu,
                bc_value=w.bc_value)
    args.update(overrides)
    return md.Problem(**args)
