"""object_scores (§6.4) on the GPU against the oracle: per query object and
database object, the sum of its descriptors' Eq. 1 distances to their
nearest descriptor of the object (FP64 sums of exact per-object minima:
equal to the oracle's FP64 sums to rounding order), +inf for objects without
descriptors, 0 for query objects without descriptors."""
import numpy as np
import pytest
import torch

import oracle
from helpers import to_dev
from paper_2107_03368_gb300 import dt, synth

pytestmark = pytest.mark.gpu


def _check(db, obj, n_obj, qd, off):
    got = dt.object_scores(to_dev(db), torch.from_numpy(obj.astype(np.uint32).view(np.int32)).cuda(),
                           n_obj, to_dev(qd), torch.from_numpy(off).cuda()).cpu().numpy()
    exp = oracle.object_scores(db, obj, n_obj, qd, off)
    fin = np.isfinite(exp)
    assert np.array_equal(np.isfinite(got), fin)
    np.testing.assert_allclose(got[fin], exp[fin], rtol=1e-12, atol=0)
    return got


def test_uneven_queries_empty_objects_and_an_empty_query():
    seed = 31
    n_obj, per = 12, 150
    db, obj = synth.database(seed, n_obj * per, per_object=per, pool=10)
    qd, off, _ = synth.partial_queries(seed, db, n_obj, per, 7, n_min=10, n_max=140)
    off = off.copy()
    off[2] = off[1]                                   # query object 1 has no descriptors
    off = np.concatenate([off[:2], off[1:]])          # and one more empty one after it
    got = _check(db, obj, n_obj + 2, qd, off)         # objects 12 and 13 hold nothing
    assert np.all(got[1] == 0) and np.all(np.isinf(got[0, n_obj:]))


def test_object_ids_in_any_order():
    rng = np.random.default_rng(3)
    db, _ = synth.database(32, 2000, per_object=200, pool=10)
    obj = rng.integers(0, 9, size=db.shape[0]).astype(np.uint32)
    obj[rng.integers(0, db.shape[0], size=50)] = 1000   # ids past n_objects are ignored
    qd, _ = synth.queries(33, db, 300)
    off = np.array([0, 1, 40, 41, 300], dtype=np.int64)
    _check(db, obj, 9, qd, off)


def test_many_objects_split_the_queries_into_chunks():
    """100,000 (mostly empty) objects: the per-object minima of ~1,300
    descriptors fill the chunk budget, so 3,000 descriptors take 3 chunks."""
    rng = np.random.default_rng(4)
    db, _ = synth.database(34, 3000, per_object=300, pool=10)
    obj = rng.integers(0, 100_000, size=db.shape[0]).astype(np.uint32)
    obj[:1500] = rng.integers(0, 40, size=1500)
    qd, _ = synth.queries(35, db, 3000)
    off = np.array([0, 900, 1000, 2200, 2999, 3000], dtype=np.int64)
    _check(db, obj, 100_000, qd, off)
