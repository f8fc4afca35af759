"""The seeded input generators: published splitmix64 vectors, ranges, determinism."""
import numpy as np

import nhmf_inputs as I


def test_splitmix64_published_vector():
    # test vector of the splitmix64 reference implementation, seed 1234567
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert I.splitmix64(1234567, 5).tolist() == ref


def test_counter_offsets_are_consistent():
    a = I.splitmix64(99, 10)
    assert np.array_equal(I.splitmix64(99, 4, offset=6), a[6:])


def test_uniform_and_normal_moments():
    u = I.uniform01(5, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 5e-3
    z = I.normal(6, 200001)
    assert z.size == 200001 and abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2


def test_workload_sizes():
    w = I.WORKLOADS["q2_64_clamp"]
    assert w.n_dofs == 6440067 and w.n_qp == 64 ** 3 * 27
    assert I.WORKLOADS["q4_32_clamp"].n_dofs == 6440067
    assert I.WORKLOADS["q1_8_clamp"].n_dofs == 2187
    assert I.WORKLOADS["q3_48_compress"].n_dofs == 9145875
    assert I.WORKLOADS["q4_64_compress"].n_dofs == 50923779


def test_draws_respect_dirichlet_and_scale():
    w = I.small(I.WORKLOADS["q2_64_clamp"], 6)
    u = I.draw_u(w)
    mask = I.dirichlet_mask(w.n_el, w.degree, w.bc).reshape(-1)
    assert np.all(u[mask] == 0.0)
    assert np.abs(u).max() <= 0.05 / (w.n_el * w.degree)
    du = I.draw_du(w)
    assert np.all(du[mask] == 0.0)
    assert np.array_equal(I.draw_u(w), u)
