"""gt_word_count_noalloc (word count with a fixed device scratch array, no
allocation) gives the same counts as gt_word_count, on two calls in a row."""
import numpy as np
import pytest
import torch

from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import sequitur, make_corpus
from tests.test_oracle_pins import tiny_cases, grammar_from_rules

pytestmark = pytest.mark.gpu


def grammars():
    out = [(n, g) for n, g, _, _ in tiny_cases(seed=91, count=6)]
    c = make_corpus("wc_single_200k")
    out.append(("wc200k", sequitur(c.tokens, c.file_lens, c.num_words)))
    m = make_corpus("multi64_50m", scale=0.004)
    out.append(("multi200k", sequitur(m.tokens, m.file_lens, m.num_words)))
    out.append(("all_empty", grammar_from_rules(5, [[], [0, 1]], [0, 0, 0])))
    return out


GRAMMARS = grammars()


@pytest.mark.parametrize("name,g", GRAMMARS, ids=[n for n, _ in GRAMMARS])
def test_noalloc_matches_word_count(name, g):
    ctx = B.gt_create(0)
    try:
        gh = B.gt_load_grammar(ctx, g)
        want = torch.full((g.num_words,), -1, dtype=torch.int64, device="cuda")
        B.gt_word_count(gh, want)
        B.gt_sync(ctx)
        for call in range(2):
            got = torch.full((g.num_words,), -7, dtype=torch.int64, device="cuda")
            B.gt_word_count_noalloc(gh, got)
            B.gt_sync(ctx)
            assert torch.equal(got, want), call  # integer counts: exact
        B.gt_free_grammar(gh)
    finally:
        B.gt_destroy(ctx)
