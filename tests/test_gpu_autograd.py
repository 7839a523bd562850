"""The differentiable projection (autograd.project) against the oracle's forward and adjoint.

The autograd op keeps one multigrid context per grid and saves p with references to its
inputs phi and the solid mask (the face coefficients are formed again in backward when the
context no longer holds them); these tests check that a backward uses its own forward's
coefficients and hierarchy also when other forwards on the same grid ran in between (the
pattern of a Runge-Kutta step with two projections, or of a batch of projections on one grid),
and that nothing but p is stored for backward.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1410_2240_gb300 import synth

from _gpu_util import dev, faces_dev, host, rel

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def ag():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_2240_gb300 import autograd
    autograd.clear_cache()
    yield autograd
    autograd.clear_cache()


def _leaf(case):
    phi = dev(case.phi).requires_grad_(True)
    u = tuple(x.requires_grad_(True) for x in faces_dev(case.u_star))
    solid = None if case.solid is None else dev(case.solid, torch.uint8)
    return phi, u, solid


def _oracle_grads(case):
    """Gradients of L = <w, P u*> with respect to u* and phi, by the oracle (FP64)."""
    _, po, beta_o, _ = O.project(case.phi, case.solid, case.u_star, case.h, lam=case.lam, tol=1e-13)
    g_u, _, g_phi = O.project_adjoint(beta_o, po, case.w, case.h, lam=case.lam, tol=1e-13)
    return g_u, g_phi


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_interleaved_forwards_each_backward_uses_its_own_hierarchy(ag, prec):
    a = synth.small_case(32, seed=1, solid="ellipsoid")
    b = synth.small_case(32, seed=2, interface="flat")
    phi_a, u_a, s_a = _leaf(a)
    phi_b, u_b, s_b = _leaf(b)
    # both forwards first (the context's hierarchy then belongs to b), then one backward
    # through both graphs: a's backward must rebuild a's hierarchy from a's coefficients
    ua, _ = ag.project(u_a, phi_a, a.h, solid=s_a, rho_air=a.lam, tol=TOL, precision=prec)
    ub, _ = ag.project(u_b, phi_b, b.h, solid=s_b, rho_air=b.lam, tol=TOL, precision=prec)
    wa, wb = faces_dev(a.w), faces_dev(b.w)
    loss = sum((x * w).sum() for x, w in zip(ua, wa)) + sum((x * w).sum() for x, w in zip(ub, wb))
    loss.backward()
    for case, phi, u in ((a, phi_a, u_a), (b, phi_b, u_b)):
        g_u, g_phi = _oracle_grads(case)
        assert rel(host(phi.grad), g_phi) <= 1e-8, case.name
        for x, gx in zip(u, g_u):
            assert rel(host(x.grad), gx) <= 1e-8, case.name


def test_repeated_steps_give_identical_gradients(ag):
    """Forward + backward twice on the same inputs: the cached context is reused without a
    rebuild in backward, and the results are the same bits."""
    case = synth.small_case(32, seed=3, solid="wall")
    grads = []
    for _ in range(2):
        phi, u, solid = _leaf(case)
        ux, _ = ag.project(u, phi, case.h, solid=solid, rho_air=case.lam, tol=TOL, precision="mixed")
        torch.autograd.backward(ux, faces_dev(case.w))
        grads.append([host(phi.grad)] + [host(x.grad) for x in u])
    for g0, g1 in zip(*grads):
        assert np.array_equal(g0, g1)


def test_saves_only_p_beside_its_inputs(ag):
    """The graph holds phi (the caller's tensor itself), the solid mask and p: one array of the
    grid's size per projection, not the face coefficients or the hierarchy."""
    case = synth.small_case(16, seed=4, solid="ellipsoid")
    phi, u, solid = _leaf(case)
    (ux, uy, uz), p = ag.project(u, phi, case.h, solid=solid, rho_air=case.lam, tol=TOL, precision="mixed")
    saved = ux.grad_fn.saved_tensors
    assert len(saved) == 3
    assert saved[0].data_ptr() == phi.data_ptr() and saved[1].data_ptr() == solid.data_ptr()
    assert saved[2].data_ptr() == p.data_ptr()
