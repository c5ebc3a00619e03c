"""Pins for the oracle's vector-scaling task (Section 2 example:
every element of the buffer is multiplied by the factor)."""
import numpy as np
import pytest

import synth


def test_power_of_two_chain_is_exact_product(orc):
    # With power-of-two factors and no over/underflow every multiply is
    # exact, so the chain equals x * prod(f) exactly.
    x = synth.vector_f32(1 << 12, seed=11)
    fs = [2.0, 0.5, 4.0, 0.25, 8.0, 2.0, 0.5, 0.125]
    y = x.copy()
    for f in fs:
        orc.tiles.scal_f32(y, f)
    assert np.array_equal(y, x * np.float32(np.prod(fs)))


def test_chain_matches_inorder_numpy_and_not_folded(orc):
    x = synth.vector_f32(1 << 16, seed=12)
    fs = synth.chain_factors(1, 8, seed=13)[0]
    y = x.copy()
    z = x.copy()
    for f in fs:
        orc.tiles.scal_f32(y, f)
        z *= np.float32(f)           # numpy binary32 multiply, one rounding
    assert np.array_equal(y.view(np.uint32), z.view(np.uint32))
    folded = x * np.float32(np.prod(fs.astype(np.float64)))
    # a folded chain rounds differently somewhere: the oracle must not fold
    assert not np.array_equal(y, folded)


def test_subnormals_are_honoured(orc):
    x = np.array([1e-38, 3e-39, -5e-45, 1.17e-38], dtype=np.float32)
    y = x.copy()
    orc.tiles.scal_f32(y, 0.5)
    z = x * np.float32(0.5)
    assert np.array_equal(y.view(np.uint32), z.view(np.uint32))
    assert y[1] != 0.0 and y[2] != 0.0


def test_executor_runs_in_submission_order_and_checks(orc):
    ex = orc.executor.Executor()
    R, W, RW = 1, 2, 3
    cl = ex.task_decl("scale_vector", orc.executor.scal_body, [RW])
    x = np.ones(8, dtype=np.float32)
    h = ex.data_register(x)
    ex.task_submit(cl, [h], scalars=(3.0,))
    ex.task_submit(cl, [h], scalars=(0.5,))
    assert np.all(x == np.float32(1.5))
    assert ex.data_lookup(x) == h
    with pytest.raises(orc.executor.OracleError) as e:
        ex.data_lookup(np.ones(3, dtype=np.float32))
    assert e.value.code == orc.executor.ENOENT
    with pytest.raises(orc.executor.OracleError) as e:
        ex.task_submit(cl, [h], modes=[R], scalars=(1.0,))
    assert e.value.code == orc.executor.EINVAL
