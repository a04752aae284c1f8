"""bench.py's copy of the paper's Tables 1-4 (the second benchmark's reference
numbers) agrees with the cited golden fixture."""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_paper_tables_match_golden():
    import bench
    rows = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_tables.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[(int(f[1]), int(f[2]))] = (float(f[5]), float(f[7]))
    assert len(bench.PAPER_TABLES) == len(rows)
    for m, n, tr, er in bench.PAPER_TABLES:
        assert rows[(m, n)] == (tr, er)
