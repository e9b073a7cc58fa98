"""The seeded generator: determinism, stated symmetries and exactness of the integrals."""
import numpy as np

import synth


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: first outputs of the published generator.
    s0 = np.uint64(0)
    n = np.arange(1, 4, dtype=np.uint64)
    with np.errstate(over="ignore"):
        out = synth._mix(s0 + n * synth._GOLDEN)
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_determinism_and_counter_access():
    a = synth.normal(7, 3, 0, 100)
    b = synth.normal(7, 3, 40, 20)
    np.testing.assert_array_equal(a[40:60], b)
    assert not np.array_equal(a, synth.normal(8, 3, 0, 100))


def test_job_symmetries_and_ranges():
    amp = synth.make_amplitudes(4, 9, 5)
    o = amp.o
    assert np.all(np.diff(amp.eps[:o]) >= 0) and np.all(np.diff(amp.eps[o:]) >= 0)
    assert amp.eps[:o].min() >= -1.5 and amp.eps[:o].max() <= -0.3
    assert amp.eps[o:].min() >= 0.1 and amp.eps[o:].max() <= 3.0
    np.testing.assert_array_equal(amp.B, amp.B.transpose(0, 2, 1))
    np.testing.assert_array_equal(amp.t2, amp.t2.transpose(1, 0, 3, 2))
    assert np.all(np.rint(amp.B * 2 ** 20) == amp.B * 2 ** 20)
    assert amp.Q == 3 * (4 + 9)


def test_integrals_are_exact_in_any_order():
    amp = synth.make_amplitudes(3, 7, 9)
    g = synth.ovvv(amp)
    # reversed-order accumulation over Q gives the same bits
    o, v = amp.o, amp.v
    acc = np.zeros_like(g)
    for q in reversed(range(amp.Q)):
        acc += np.einsum("ia,bd->iabd", amp.B[q, :o, o:], amp.B[q, o:, o:])
    np.testing.assert_array_equal(acc, g)
    np.testing.assert_array_equal(g, g.transpose(0, 1, 3, 2))
    np.testing.assert_array_equal(synth.ovvv_slice(amp, 2), g[2])
    ov = synth.ovov(amp)
    np.testing.assert_array_equal(ov, ov.transpose(2, 3, 0, 1))


def test_serving_shapes_in_range():
    for r in range(200):
        o, v = synth.serving_request_shape(r)
        assert 6 <= o <= 32 and 6 * o - 1 <= v <= 12 * o + 1


def test_device_generator_twin_matches_host_generator():
    """The torch twin (run here on the CPU) draws the same uniforms bit for bit;
    normals agree to the last place (log/cos of another math library), and the
    factor values, rounded to the 2^-20 grid, agree exactly on these shapes."""
    import torch
    for (o, v, seed) in [(3, 7, 5), (4, 11, synth.SERVING_SEED_BASE + 7)]:
        assert np.array_equal(synth.uniform(seed, 5, 3, 200), synth.uniform_t(seed, 5, 3, 200, "cpu").numpy())
        a = synth.make_amplitudes(o, v, seed)
        b = synth.make_amplitudes_device(o, v, seed, device="cpu")
        assert np.array_equal(a.eps, b["eps"].numpy())
        assert np.array_equal(a.B, b["B"].numpy())
        assert np.allclose(a.t1, b["t1"].numpy(), rtol=1e-14, atol=0)
        assert np.allclose(a.t2, b["t2"].numpy(), rtol=1e-13, atol=1e-20)
        d = synth.device_job_from_factor(b)
        assert np.array_equal(d["ovoo"].numpy(), synth.ovoo(a))
        assert torch.equal(d["ovov"], torch.from_numpy(synth.ovov(a)))
