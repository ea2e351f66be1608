"""dt_save / dt_load on the GPU: a built tree and a tree grown by dt_insert
come back identical (nodes, images, permutation, shape), and searches on the
loaded index equal searches on the saved one and the oracle."""
import numpy as np
import pytest
import torch

from helpers import assert_matches_oracle, edge_queries, mixed_db, to_dev
from paper_2107_03368_gb300 import dt

pytestmark = pytest.mark.gpu


def same_index(a, b, with_and):
    ea, eb = a.export(with_and=with_and), b.export(with_and=with_and)
    for f in ea:
        if ea[f] is not None:
            assert np.array_equal(ea[f], eb[f]), f
    assert a.info() == b.info()


@pytest.mark.parametrize("grown,use_and", [(False, False), (False, True), (True, True)])
def test_save_load_roundtrip(tmp_path, grown, use_and):
    db = mixed_db(71, 6000)
    d_db = to_dev(db)
    if grown:
        ix = dt.dt_build(to_dev(db[:4000]), leaf_size=16, use_and_image=use_and)
        dt.dt_insert(ix, to_dev(db[4000:]))
    else:
        ix = dt.dt_build(d_db, leaf_size=16, use_and_image=use_and)
    path = tmp_path / "tree.dtix"
    ix.save(path)
    back = dt.dt_load(path, d_db)
    same_index(ix, back, use_and)
    q = edge_queries(72, db, 60)
    d_q = to_dev(q)
    a = dt.dt_search(ix, d_q, 7, with_ab=True)
    b = dt.dt_search(back, d_q, 7, with_ab=True)
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    assert_matches_oracle(db, q, 7, *b[:3])
    with pytest.raises(dt.DtError) as e:
        dt.dt_load(path, d_db[:5000].contiguous())
    assert e.value.status == dt.DT_EINVAL
    ix.free()
    back.free()


def test_load_over_other_rows_is_rejected(tmp_path):
    """The file keeps the images, not the descriptors: loading it over a
    database of the same size but other contents (here the same rows in
    another order, and one row set to all ones) must be refused, since its images
    would no longer bound their subtrees."""
    db = mixed_db(73, 3000)
    d_db = to_dev(db)
    ix = dt.dt_build(d_db, leaf_size=16, use_and_image=True)
    path = tmp_path / "tree.dtix"
    ix.save(path)
    rng = np.random.default_rng(0)
    changed = db.copy()
    changed[1234] = np.uint64(0xFFFFFFFFFFFFFFFF)     # widens its leaf's OR image
    for other in (db[rng.permutation(db.shape[0])], changed):
        with pytest.raises(dt.DtError) as e:
            dt.dt_load(path, to_dev(other))
        assert e.value.status == dt.DT_EINVAL
        assert "images" in dt.dt_last_error()
    back = dt.dt_load(path, d_db)          # the right rows still load
    assert back.info() == ix.info()
    ix.free()
    back.free()

