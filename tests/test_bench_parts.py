"""bench.py's e2e step classifies the reads in parts (one mc_classify call
per part): the parts must cover every query, mate and base exactly once,
in order, with offsets that reproduce the original ones."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_read_parts_partition_the_queries():
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(5)
    nq = 1003
    mates = rng.integers(1, 3, nq)                      # single-end and pairs
    qoffs = np.concatenate([[0], np.cumsum(mates)]).astype(np.uint32)
    lens = rng.integers(0, 300, int(qoffs[-1]))         # empty mates included
    roffs = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    for n_parts in (1, 2, 4, 7):
        parts = bench.read_parts(roffs, qoffs, n_parts)
        assert len(parts) == n_parts
        assert parts[0][0] == 0 and parts[-1][1] == nq
        for (qa, qb, nm, ba, bb, ro, qo), nxt in zip(parts, parts[1:] + [None]):
            if nxt is not None:
                assert nxt[0] == qb and nxt[3] == bb
            assert ro.dtype == np.uint64 and qo.dtype == np.uint32
            assert qo[0] == 0 and ro[0] == 0 and len(qo) == qb - qa + 1 and len(ro) == nm + 1
            assert (qo.astype(np.int64) + int(qoffs[qa]) == qoffs[qa:qb + 1]).all()
            ma = int(qoffs[qa])
            assert (ro + np.uint64(ba) == roffs[ma:ma + nm + 1]).all()
            assert ba == int(roffs[ma]) and bb == int(roffs[ma + nm])
