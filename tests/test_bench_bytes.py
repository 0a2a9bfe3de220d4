"""Host-side arithmetic of bench.py: the root layout the chunk sort works on
and the algorithmic bytes each timed kernel is credited with."""
import sys
from pathlib import Path
from types import SimpleNamespace

import numpy as np

sys.path.insert(0, str(Path(__file__).resolve().parent.parent))
import bench  # noqa: E402


def test_root_layout_counts_file_pure_chunks():
    # files of 0, 1, 8192, 8193 and 20000 root symbols: 0 + 1 + 1 + 2 + 3 chunks
    lens = [0, 1, 8192, 8193, 20000]
    file_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    g = SimpleNamespace(file_off=file_off, rule_off=np.array([0, file_off[-1], file_off[-1] + 2], np.int64))
    lay = bench.root_layout(g)
    assert lay == {"root_len": sum(lens), "root_chunks": 7}


def test_algorithmic_bytes_per_kernel():
    info = {"num_syms": 1000, "num_words": 500_000, "num_files": 64, "root_words": 300, "file_words": 50,
            "file_pairs": 20}
    root = {"root_len": 400, "root_chunks": 3}
    ab = bench.algorithmic_bytes(info, tv_entries=70, root=root)
    nb = 31  # 500,000 words in buckets of 2^14
    assert ab["wc_partition"] == ("wc_partition_kernel", 4 * 1000)
    assert ab["tv_hist_kernel"] == ("tv_hist_kernel", 2 * 300 + 8 * 50 + 8 * 70 + 2056 * 64 * nb)
    # the root chunk sort's kernel name carries the bucket index width (5 bits for 31 buckets)
    assert ab["chunk_sort_root"] == ("chunk_sort_kernel<0, 5>", 4 * 400 + 2 * 300 + 12 * 3 * nb)
    assert ab["expand_words"] == ("expand_words_kernel", 36 * 20 + 12 * 50)


def test_bucket_index_width_matches_the_launch_dispatch():
    # width = bits of (nb - 1), 0 for a single bucket, as the launcher computes it
    for V, bits in ((1, 0), (16384, 0), (16385, 1), (32768, 1), (49152, 2), (500_000, 5), (1 << 21, 7)):
        info = {"num_syms": 0, "num_words": V, "num_files": 1, "root_words": 0, "file_words": 0, "file_pairs": 0}
        name = bench.algorithmic_bytes(info, 0, {"root_len": 0, "root_chunks": 0})["chunk_sort_root"][0]
        assert name == f"chunk_sort_kernel<0, {bits}>", (V, name)


def test_cpu_baseline_runs_the_step_analytics_on_a_file_prefix():
    from paper_2106_06889_gb300.corpus import sequitur
    rng = np.random.default_rng(5)
    lens = np.array([400, 300, 500, 200], np.int64)
    toks = rng.integers(0, 50, size=int(lens.sum())).astype(np.int32)
    g = sequitur(toks, lens, 50)
    rate, nfiles, ntok, dt = bench.oracle_sample(g, ["word_count", "inverted_index", "term_vector"], budget_s=0.0)
    # a zero budget stops after the first prefix: one file, its tokens counted
    assert nfiles == 1 and ntok == 400 and dt > 0 and rate == ntok / dt
    rate, nfiles, ntok, dt = bench.oracle_sample(g, ["sequence_count"], budget_s=1e9)
    # an unbounded budget grows the prefix to every file
    assert nfiles == 4 and ntok == int(lens.sum())
