"""The seeded input recipes (CPU): each generator draws what the stated recipe
says, in the stated order, rounded once to complex64, and the uneven batch
reproduces the length histogram recorded with its recipe (4096 lengths 2^k,
k ~ U{6..16} from default_rng(2): sum 49,093,248, bins k = 6..16 below)."""
import numpy as np
import pytest

from paper_0811_2535_gb300 import inputs

UNEVEN_BINS = [366, 406, 404, 336, 368, 358, 389, 362, 357, 364, 386]   # k = 6..16


def test_seeds_are_the_recorded_ones():
    assert (inputs.SEED_SMALL, inputs.SEED_LARGE, inputs.SEED_UNEVEN, inputs.SEED_PRECISION,
            inputs.SEED_GRADIENT) == (0, 1, 2, 3, 4)


@pytest.mark.parametrize("shape", [(1024,), (64, 32), (4, 8, 16)])
def test_uniform_recipe(shape):
    x = inputs.uniform(shape, 7)
    rng = np.random.default_rng(7)
    re = rng.uniform(-1.0, 1.0, size=shape)
    im = rng.uniform(-1.0, 1.0, size=shape)
    assert x.dtype == np.complex64 and x.shape == shape
    assert np.array_equal(x.real, re.astype(np.float32)) and np.array_equal(x.imag, im.astype(np.float32))
    assert np.all(np.abs(x.real) <= 1) and np.all(np.abs(x.imag) <= 1)
    assert np.array_equal(inputs.uniform(shape, 7), x)              # reproducible


def test_large_workload_is_one_fresh_generator_per_shape():
    a = inputs.uniform((1 << 12,), inputs.SEED_LARGE)
    b = inputs.uniform((64, 64), inputs.SEED_LARGE)
    assert np.array_equal(a, b.reshape(-1))     # same seed, same draw order, reshaped


def test_uneven_batch_recipe_and_histogram():
    lengths, vecs = inputs.uneven_batch(4096, inputs.SEED_UNEVEN)
    k = np.log2(lengths).astype(int)
    assert np.array_equal(lengths, np.int64(1) << k)
    assert int(lengths.sum()) == 49_093_248
    assert [int((k == b).sum()) for b in range(6, 17)] == UNEVEN_BINS
    assert np.array_equal(k, inputs.uneven_lengths(4096, inputs.SEED_UNEVEN))
    # the vectors follow the lengths, re then im ~ N(0, 1), transform by transform
    rng = np.random.default_rng(inputs.SEED_UNEVEN)
    rng.integers(6, 17, 4096)
    for n, v in list(zip(lengths, vecs))[:5]:
        re = rng.standard_normal(int(n))
        im = rng.standard_normal(int(n))
        assert v.dtype == np.complex64 and v.size == n
        assert np.array_equal(v.real, re.astype(np.float32)) and np.array_equal(v.imag, im.astype(np.float32))
    allv = np.concatenate(vecs).astype(np.complex128)
    assert abs(allv.real.mean()) < 1e-3 and abs(allv.real.std() - 1) < 1e-3


def test_sinusoids_put_their_peaks_where_drawn():
    """Each transform is noise plus five sinusoids of amplitude 10 at distinct
    integer frequencies: the DFT (numpy, FP64) has bins of magnitude 10 n there
    and only noise elsewhere."""
    batch, n = 4, 256
    x = inputs.sinusoids(batch, n, inputs.SEED_PRECISION)
    assert x.dtype == np.complex64 and x.shape == (batch, n)
    rng = np.random.default_rng(inputs.SEED_PRECISION)
    rng.uniform(-1.0, 1.0, size=(batch, n))
    rng.uniform(-1.0, 1.0, size=(batch, n))
    X = np.fft.fft(x.astype(np.complex128), axis=1)
    for b in range(batch):
        f = rng.choice(n, size=5, replace=False)
        phi = rng.uniform(0.0, 1.0, size=5)
        assert len(set(f.tolist())) == 5
        # exp(+2 pi i f j / n) lands in bin f of the sign -1 transform with phase phi
        peak = X[b, f]
        assert np.allclose(np.abs(peak), 10 * n, rtol=0.02)
        assert np.allclose(np.angle(peak / np.exp(2j * np.pi * phi)), 0, atol=0.02)
        rest = np.delete(np.abs(X[b]), f)
        assert rest.max() < 0.2 * 10 * n


def test_spectral_filter_draw_order():
    n, batch = 64, 3
    H, x = inputs.spectral_filter(n, batch, inputs.SEED_GRADIENT)
    rng = np.random.default_rng(inputs.SEED_GRADIENT)
    hre, him = rng.standard_normal(n), rng.standard_normal(n)
    xre, xim = rng.uniform(-1, 1, size=(batch, n)), rng.uniform(-1, 1, size=(batch, n))
    assert H.shape == (n,) and x.shape == (batch, n)
    assert np.array_equal(H.real, hre.astype(np.float32)) and np.array_equal(H.imag, him.astype(np.float32))
    assert np.array_equal(x.real, xre.astype(np.float32)) and np.array_equal(x.imag, xim.astype(np.float32))


def test_no_transform_arithmetic_in_the_inputs_module():
    """The module imports only numpy (and __future__) and calls no FFT."""
    import ast
    import inspect
    tree = ast.parse(inspect.getsource(inputs))
    imported = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            imported.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            imported.add((node.module or "").split(".")[0])
        elif isinstance(node, ast.Attribute):
            assert node.attr != "fft", "an FFT call in the inputs module"
    assert imported <= {"numpy", "__future__"}, imported
