"""Float64 restatement of the tensor-core row pass's arithmetic (no GPU).

The tcgen05 pass computes each row's length-L convolution (Section 2.2, steps
4-8) as four real matrix products of a four-step FFT split L = R1 x 32 with
the paper's 2N padding: only n1 < R1 / 2 is nonzero on input and only
n1 < R1 / 2 is kept on output, each inverse DFT is taken as
conj(DFT(conj(.))), and every DFT matrix carries a 1/sqrt(R) scale.  These
tests restate that formulation in float64 -- with the operand packing of the
real products ([Re | Im] against [[Fr, Fi], [-Fi, Fr]]) and the row / lane
order the kernel uses -- and check it against the circular convolution of
numpy's FFT, for the three built lengths.  They also check the position-to-
frequency map by which the kernel spectrum is put in natural order (the FP32
network's radix-16 decimation-in-frequency digits), against a stage-by-stage
emulation of such a network.  They test the design's index mathematics, not
the CUDA code (the GPU tests do that against the oracle).
"""

import numpy as np
import pytest

R2 = 32


def dft(n):
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n) / np.sqrt(n)


def real_block(F, kin, nout):
    """B[(s, i)][(t, o)] of D = [Re | Im] B: the real form of x -> x F restricted to kin inputs, nout outputs."""
    f = F[:kin, :nout]
    return np.block([[f.real, f.imag], [-f.imag, f.real]])


def four_step_rows(X, Hn, L):
    """The tile arithmetic for rows X [rows, L] (zero beyond L / 2) and the natural-order spectrum
    Hn = FFT(h) / sqrt(L): returns the first L / 2 outputs of the circular convolution of each row,
    scaled by 1 / L as the kernel's output chirp expects."""
    R1 = L // R2
    KA = NA = R1 // 2
    rows = X.shape[0]
    F1, F2 = dft(R1), dft(R2)
    T = np.exp(-2j * np.pi * np.outer(np.arange(R2), np.arange(R1)) / L)  # W_L^{n2 k1}, [n2][k1]
    BA, BB, BAH = real_block(F1, KA, R1), real_block(F2, R2, R2), real_block(F1, R1, NA)
    # stage A: operand rows (r, n2), K = (re, im) of n1 < KA
    AA = np.zeros((rows * R2, 2 * KA))
    for r in range(rows):
        for n2 in range(R2):
            v = X[r, R2 * np.arange(KA) + n2]
            AA[R2 * r + n2] = np.r_[v.real, v.imag]
    DA = AA @ BA
    Y = (DA[:, :R1] + 1j * DA[:, R1:]) * np.tile(T, (rows, 1))  # rows (r, n2), columns k1
    # stage B: operand rows (r, k1) = R1 r + k1, K = n2
    AB = np.zeros((rows * R1, 2 * R2))
    for r in range(rows):
        for k1 in range(R1):
            v = Y[R2 * r:R2 * (r + 1), k1]
            AB[R1 * r + k1] = np.r_[v.real, v.imag]
    DB = AB @ BB
    S = DB[:, :R2] + 1j * DB[:, R2:]  # X[k1 + R1 k2] / sqrt(L) at row (r, k1), column k2
    W = np.empty_like(S)
    for r in range(rows):
        for k1 in range(R1):
            W[R1 * r + k1] = S[R1 * r + k1] * Hn[k1 + R1 * np.arange(R2)]
    # stage B^H: conj in, K = k2
    DBH = np.concatenate([W.real, -W.imag], axis=1) @ BB
    D = DBH[:, :R2] + 1j * DBH[:, R2:]  # rows (r, k1), columns n2
    # stage A^H: operand rows (r, n2), K = k1 (twiddle again; the conjugations cancel)
    AAH = np.zeros((rows * R2, 2 * R1))
    for r in range(rows):
        for k1 in range(R1):
            v = D[R1 * r + k1] * T[:, k1]
            AAH[R2 * r + np.arange(R2), k1] = v.real
            AAH[R2 * r + np.arange(R2), R1 + k1] = v.imag
    DAH = AAH @ BAH
    yc = DAH[:, :NA] + 1j * DAH[:, NA:]
    out = np.zeros((rows, R2 * NA), complex)
    for r in range(rows):
        for n2 in range(R2):
            out[r, R2 * np.arange(NA) + n2] = np.conj(yc[R2 * r + n2])
    # the three 1/sqrt(L) stage scales against the transform's 1/L (carried by the output chirp)
    return out * np.sqrt(L) / L


@pytest.mark.parametrize("L", [512, 1024, 2048])
def test_four_step_products_equal_the_circular_convolution(L):
    rng = np.random.default_rng(L)
    rows = 8 if L == 512 else 4  # the kernel's tile rows
    X = np.zeros((rows, L), complex)
    X[:, :L // 2] = rng.standard_normal((rows, L // 2)) + 1j * rng.standard_normal((rows, L // 2))
    h = np.exp(1j * np.pi * rng.uniform(0, 1e-3) * (np.arange(L) - L // 2) ** 2)  # any kernel
    H = np.fft.fft(h)
    ref = np.fft.ifft(np.fft.fft(X, axis=1) * H, axis=1)[:, :L // 2]
    got = four_step_rows(X, H / np.sqrt(L), L) * L  # undo the output chirp's 1/L
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-12, err


@pytest.mark.parametrize("L", [512, 1024, 2048])
def test_four_step_pruned_inputs_and_outputs(L):
    """Only n1 < R1 / 2 enters and leaves: inputs beyond L / 2 are ignored (they are the zero padding),
    and the kept outputs are exactly the first L / 2 of the circular convolution."""
    rng = np.random.default_rng(7 * L)
    X = np.zeros((4, L), complex)
    X[:, :L // 2] = rng.standard_normal((4, L // 2))
    Xdirty = X.copy()
    Xdirty[:, L // 2:] = 99.0  # would change the result if the pass read it
    H = np.fft.fft(rng.standard_normal(L) + 1j * rng.standard_normal(L))
    assert np.array_equal(four_step_rows(X, H, L), four_step_rows(Xdirty, H, L))


def dif_network(x, radices):
    """Stage-by-stage radix-R decimation-in-frequency FFT without reordering (positions in the network's
    own order), as the FP32 row pass runs it."""
    L = x.size
    v = x.astype(complex).copy()
    Mp = L
    for R in radices:
        M = Mp // R
        out = v.copy()
        k = np.arange(R)
        for K in range(L // Mp):
            for n in range(M):
                idx = K * Mp + n + k * M
                y = (np.exp(-2j * np.pi * np.outer(k, k) / R) @ v[idx]) * np.exp(-2j * np.pi * n * k / Mp)
                out[idx] = y
        v = out
        Mp = M
    return v


@pytest.mark.parametrize("L", [512, 1024, 2048, 4096])
def test_natural_order_map_of_the_radix16_network(L):
    """Position p of the network holds frequency f(p) = sum_s k_s R_0 ... R_{s-1}, with k_s = (p / M_s)
    mod R_s its stage digits (stages of radix min(M, 16)): the map that puts the kernel spectrum in the
    natural order the tensor-core pass indexes, a permutation of 0 .. L-1."""
    radices, M = [], L
    while M > 1:
        R = min(M, 16)
        radices.append(R)
        M //= R
    x = np.random.default_rng(L).standard_normal(L) + 1j * np.random.default_rng(L + 1).standard_normal(L)
    v = dif_network(x, radices)
    f = np.zeros(L, int)
    for p in range(L):
        Ms, w, acc = L, 1, 0
        for R in radices:
            Ms //= R
            acc += ((p // Ms) % R) * w
            w *= R
        f[p] = acc
    assert np.array_equal(np.sort(f), np.arange(L))
    assert np.allclose(v, np.fft.fft(x)[f], rtol=0, atol=1e-9 * np.abs(x).sum())
