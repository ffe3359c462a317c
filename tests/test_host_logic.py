"""Host-side logic without a GPU: input generators for uneven domains, the
embedding of a domain in a larger periodic box, and the padded-side candidates."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2403_19854_gb300 import workloads as W


def test_embed_keeps_domain_and_zero_pads():
    p = W.spheres_problem(n_box=16, n_spheres=2, a_tilde=2.5, degree=1, r_range=(0.2, 0.3), seed=3)
    q = W.embed(p, (20, 18, 24))
    assert q.n == (20, 18, 24) and q.h == p.h
    c3 = q.chi.reshape(24, 18, 20)
    assert np.array_equal(c3[:16, :16, :16].reshape(-1), p.chi)
    assert c3.sum() == p.chi.sum()
    assert np.all(q.V.reshape(24, 18, 20)[16:] == 0) and np.all(q.r.reshape(24, 18, 20)[:, :, 16:] == 0)
    with pytest.raises(ValueError):
        W.embed(p, (15, 16, 16))


def test_embedding_is_invisible_to_the_oracle():
    """The stiffness action on the domain's nodes does not depend on the periodic box
    around it once the gap of Eq. 66 holds (translation invariance, Eq. 71)."""
    p = W.spheres_problem(n_box=16, n_spheres=1, a_tilde=2.5, degree=1, r_range=(0.2, 0.25), seed=9)
    q = W.embed(p, (20, 17, 18))
    d = W.random_field(p.nbox, 1) * p.chi
    dq = W.embed(W.Problem(n=p.n, h=p.h, a_tilde=2.5, degree=1, chi=p.chi, chi_gamma=p.chi_gamma, V=p.V,
                           r=d, g=p.g), q.n).r
    f = Oracle(p.n, p.h, 2.5, 1, p.chi).apply_K(p.V, d)
    fq = Oracle(q.n, q.h, 2.5, 1, q.chi).apply_K(q.V, dq)
    assert np.allclose(fq[q.chi > 0], f[p.chi > 0], rtol=0, atol=1e-13 * np.abs(f).max())


def test_batched_domains_seeded_and_shaped():
    a = W.batched_domains(n_domains=3, side_range=(16, 24), n_rhs=2, seed=7)
    b = W.batched_domains(n_domains=3, side_range=(16, 24), n_rhs=2, seed=7)
    for (p, rp), (q, rq) in zip(a, b):
        assert p.n == q.n and np.array_equal(p.chi, q.chi)
        assert all(np.array_equal(x, y) for x, y in zip(rp, rq))
        assert 16 <= p.n[0] <= 24 and p.degree in (1, 2)
        assert p.a_tilde == (2.5 if p.degree == 1 else 3.0)
        assert len(rp) == 2 and all(np.all(r[p.chi == 0] == 0) for r in rp)
        assert p.n_omega > 0
