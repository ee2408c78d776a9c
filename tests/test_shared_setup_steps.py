"""The integer steps by which two lanes share a chirp's run set-up (render kernel, partner_state):
moving a run's 32-bit cascade state (p, f, g; third difference zero) forward by one run of 32
samples is p + 32 f + 496 g, f + 32 g, and backward p - 32 f + 528 g, f - 32 g.  Checked here
against the cascade itself (p += f, f += g per sample, mod 2^32) on random states; the GPU tests
check the render's output against the oracle."""
import numpy as np

M = 1 << 32


def cascade(p, f, g, steps):
    for _ in range(steps):
        p = (p + f) % M
        f = (f + g) % M
    return p, f


def forward(p, f, g):
    return (p + 32 * f + 496 * g) % M, (f + 32 * g) % M


def backward(p, f, g):
    return (p - 32 * f + 528 * g) % M, (f - 32 * g) % M


def test_forward_step_is_32_cascade_steps():
    rng = np.random.default_rng(5)
    for _ in range(200):
        p, f, g = (int(v) for v in rng.integers(0, M, 3))
        assert forward(p, f, g) == cascade(p, f, g, 32)


def test_backward_step_inverts_the_forward_one():
    rng = np.random.default_rng(6)
    for _ in range(200):
        p, f, g = (int(v) for v in rng.integers(0, M, 3))
        q, h = cascade(p, f, g, 32)
        assert backward(q, h, g) == (p, f)
        # and the backward state continued for r samples is the forward one's sample r - 32 ... r
        for r in (0, 1, 17, 31):
            assert cascade(*backward(q, h, g), g, r)[0] == cascade(p, f, g, r)[0]


def test_step_constants_are_the_binomials():
    # C(32, 2) = 496 forward, C(-32, 2) = (-32)(-33)/2 = 528 backward
    assert 32 * 31 // 2 == 496 and (-32) * (-33) // 2 == 528
