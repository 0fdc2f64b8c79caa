"""Static check of the CUDA sources (CPU only): every device wait is bounded.
The only spin loop is the mbarrier wait, which gives up after kWaitCycles
clocks; no other loop in the sources spins on memory, and the mbarrier's
try_wait is issued only through it.  A new loop fails this test until it is
reviewed and listed here."""

import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2204_13393_gb300", "csrc")

# the while loops of the sources, reviewed: (file, loop text)
REVIEWED_WHILE = {
    ("lo_umma.cu", "while (!mbar_try(mb, parity))"),   # bounded by clock64() - t0 > kWaitCycles
    # the same wait, which also returns when another role of the CTA set its abort word
    ("lo_umma.cu", "while (!mbar_try(mb, parity)) {"),
    ("lo_api.cu", "while (c0 < Kmax) c0 *= 2;"),        # host: chunk-size candidates
    # host: the Householder sub-tile rows, halving from 2^14 (at most 14 steps)
    ("lo_internal.h", "while (T > s && (int64_t)(T + s) * s * 8 > kHHTileBytes) T >>= 1;"),
    # the persistent batched launch: its flag wait, bounded by kBatchWaitCycles and the abort word
    ("lo_kernels.cu", "while (ld_acquire(p) < v) {"),
    # item decoding: at most kBatchPhases phases and ninst instances (g < the list's end)
    ("lo_kernels.cu", "while (g >= pref[ph * (ninst + 1) + ninst]) ++ph;"),
    ("lo_kernels.cu", "while (g >= pref[ph * (ninst + 1) + j + 1]) ++j;"),
}


def sources():
    for fn in sorted(os.listdir(CSRC)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, fn)) as f:
                yield fn, f.read()


def code_lines(text):
    for line in text.splitlines():
        line = line.split("//")[0].strip()
        if line:
            yield line


def test_every_while_loop_is_reviewed():
    found = set()
    for fn, text in sources():
        for line in code_lines(text):
            if re.search(r"\bwhile\s*\(", line):
                found.add((fn, line))
    assert found == REVIEWED_WHILE, found ^ REVIEWED_WHILE


def test_no_endless_for_or_do_loops():
    for fn, text in sources():
        for line in code_lines(text):
            assert not re.search(r"\bfor\s*\(\s*;\s*;\s*\)", line), (fn, line)
            assert not re.search(r"\bdo\s*\{", line), (fn, line)


def test_mbarrier_wait_is_bounded_and_the_only_try_wait():
    text = dict(sources())["lo_umma.cu"]
    body = re.search(r"bool mbar_wait\(uint32_t mb, uint32_t parity\) \{(.*?)\n\}", text, re.S).group(1)
    assert "clock64() - t0 > kWaitCycles" in body and "return false" in body
    live = re.search(r"bool mbar_wait_live\(uint32_t mb, uint32_t parity, const int\* abort\) \{(.*?)\n\}", text,
                     re.S).group(1)
    assert "clock64() - t0 > kWaitCycles) return false;" in live and "abort)) return false;" in live
    assert re.search(r"constexpr long long kWaitCycles = \d+ll;", text)
    for fn, t in sources():
        hits = [l for l in code_lines(t) if "try_wait" in l]
        assert len(hits) == (1 if fn == "lo_umma.cu" else 0), (fn, hits)
        calls = [l for l in code_lines(t) if "mbar_try(" in l and "bool mbar_try(" not in l]
        want = (["if (mbar_try(mb, parity)) return true;", "while (!mbar_try(mb, parity))",
                 "if (mbar_try(mb, parity)) return true;", "while (!mbar_try(mb, parity)) {"]
                if fn == "lo_umma.cu" else [])
        assert calls == want, (fn, calls)  # mbar_try only inside the two bounded waits


def test_batch_flag_wait_is_bounded():
    """The persistent batched launch's only spin: it gives up after
    kBatchWaitCycles clocks (latching LO_ERR_TIMEOUT and the batch's abort
    word) or as soon as another CTA has aborted; its item loop is bounded by
    the number of items."""
    text = dict(sources())["lo_kernels.cu"]
    body = re.search(r"bool batch_wait\(const int\* p, int v, int\* abort_word, int\* flags\) \{(.*?)\n\}", text,
                     re.S).group(1)
    assert "clock64() - t0 > kBatchWaitCycles" in body and "break" in body
    assert "ld_acquire(abort_word) != 0" in body and "LO_ERR_TIMEOUT" in body
    assert re.search(r"constexpr long long kBatchWaitCycles = \d+ll;", text)
    assert "for (int pass_no = 0; pass_no <= total; ++pass_no)" in text
