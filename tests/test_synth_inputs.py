"""The seeded input generator (csrc/synth.c) keeps the recipe the inputs are
described by: seeded and thread-count independent, rows regenerable one by
one, object ids i // per_object, about 6% of bits set, queries made by
clearing set bits with p = 0.30 and then flipping every bit with p = 0.005,
partial-object queries as contiguous runs of one object's rows."""
import numpy as np

from paper_2107_03368_gb300 import synth


def _popc(a):
    return np.unpackbits(np.ascontiguousarray(a).view(np.uint8), axis=-1).sum(axis=-1)


def test_database_is_seeded_and_rows_regenerate_alone():
    db, obj = synth.database(5, 3000, per_object=100, nthreads=4)
    db1, obj1 = synth.database(5, 3000, per_object=100, nthreads=1)
    assert np.array_equal(db, db1) and np.array_equal(obj, obj1)
    assert np.array_equal(obj, np.arange(3000) // 100)
    for i in (0, 99, 100, 1234, 2999):
        assert np.array_equal(synth.descriptor(5, i, per_object=100), db[i])
    other, _ = synth.database(6, 3000, per_object=100)
    assert not np.array_equal(db, other)


def test_database_density_and_object_structure():
    db, obj = synth.database(7, 20_000, per_object=1000, nthreads=8)
    frac = _popc(db) / 4096.0
    assert 0.05 < frac.mean() < 0.07, frac.mean()
    assert np.mean(frac < 0.02) < 0.01
    assert np.mean(frac > 0.10) < 0.04
    # rows of one object are jittered copies of its curve sets: a row
    # shares far more set bits with its own object's rows than with others'
    rng = np.random.default_rng(0)
    rows = rng.choice(20_000, 200, replace=False)
    same, diff = [], []
    for i in rows:
        o = obj[i]
        mates = db[o * 1000:(o + 1) * 1000]
        strangers = db[((o + 1) % 20) * 1000:((o + 1) % 20 + 1) * 1000]
        same.append(np.sort(_popc(mates & db[i]))[-2])     # the best mate other than itself
        diff.append(_popc(strangers & db[i]).max())
    assert np.mean(np.array(same) > np.array(diff)) > 0.95


def test_queries_clear_then_flip_at_the_stated_rates():
    db, _ = synth.database(8, 5000, per_object=500, nthreads=8)
    q, src = synth.queries(9, db, 3000, nthreads=8)
    assert src.min() >= 0 and src.max() < 5000
    s = db[src]
    set_bits = _popc(s).sum()
    kept = _popc(q & s).sum() / set_bits
    turned_on = _popc(q & ~s).sum() / (4096.0 * len(q) - set_bits)
    # a set bit survives the clearing (0.7) and then its flip (0.995), or is
    # cleared (0.3) and flipped back on (0.005)
    assert abs(kept - (0.7 * 0.995 + 0.3 * 0.005)) < 0.004, kept
    assert abs(turned_on - 0.005) < 0.0003, turned_on
    clean, src2 = synth.queries(9, db, 50, p_clear=0.0, p_flip=0.0)
    assert np.array_equal(clean, db[src2])


def test_partial_queries_are_contiguous_runs_of_one_object():
    per, n_obj = 200, 12
    db, _ = synth.database(10, per * n_obj, per_object=per)
    qd, off, qobj = synth.partial_queries(11, db, n_obj, per, 40, n_min=20, n_max=60,
                                          p_clear=0.0, p_flip=0.0)
    counts = np.diff(off)
    assert off[0] == 0 and off[-1] == qd.shape[0]
    assert counts.min() >= 20 and counts.max() <= 60
    assert qobj.min() >= 0 and qobj.max() < n_obj
    for q in range(40):
        rows = db[qobj[q] * per:(qobj[q] + 1) * per]
        run = qd[off[q]:off[q + 1]]
        starts = [st for st in range(per - len(run) + 1) if np.array_equal(rows[st], run[0])]
        assert any(np.array_equal(rows[st:st + len(run)], run) for st in starts), q
