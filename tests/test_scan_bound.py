"""CPU check of the pass bound of the edge scan (edge_core.cuh, scan_pass_cap
and edge_scan): a pass-by-pass model of the scan's state machine, driven by
random verdicts (end probes, interior probes, witness probes, verification
batches), never needs more passes than the bound with which the kernel
stops a scan that would not progress.  The model follows the kernel's
transitions: the split once per staged edge, per chunk of 32 durations the
end probe, then interior probes (packed: the lowest eight unprobed
survivors x four samples in one pass; otherwise one sample per pass) and
verification of the lowest probed survivor, a witness pass after each
failed verification in witness mode 2."""
import numpy as np
import pytest


def scan_pass_cap(n, S):
    return ((n + 31) // 32 + 1) * (2 + 32 * (5 + (S + 31) // 32)) + 2


def lowest_bits(x, n):
    r = 0
    for _ in range(n):
        if not x:
            break
        b = x & -x
        r |= b
        x ^= b
    return r


def model_passes(rng, Kadm, S, wmode, p_end, p_mid, p_ver):
    """Passes of one grid-mode scan over [0, Kadm) with random verdicts."""
    passes = 1                                 # the split
    packed = wmode == 0
    nb = (S + 31) // 32
    for base in range(0, Kadm, 32):
        passes += 1                            # end probe
        n = min(32, Kadm - base)
        cand = sum(1 << i for i in range(n) if rng.random() < p_end)
        mpr = 0 if S > 2 else (1 << 32) - 1
        if cand and wmode == 2 and base == 0:  # the caller's witness
            passes += 1
            cand &= sum(1 << i for i in range(32) if rng.random() < p_mid)
        while cand:
            low = (cand & -cand).bit_length() - 1
            if (mpr >> low) & 1:               # verify the lowest survivor
                ok = True
                for _ in range(nb):
                    passes += 1
                    if rng.random() >= p_ver:
                        ok = False
                        break
                if ok:
                    return passes
                cand &= ~(1 << low)
                if cand and wmode == 2:        # witness pass at the rest
                    passes += 1
                    cand &= sum(1 << i for i in range(32) if rng.random() < p_mid)
                continue
            if packed:
                sel = lowest_bits(cand & ~mpr, 8)
                passes += 1
                failed = sum(1 << i for i in range(32) if (sel >> i) & 1 and rng.random() >= p_mid)
                cand &= ~failed
                mpr |= sel
            else:
                sel = cand & ~mpr
                for _ in range(4):
                    passes += 1
                    cand &= ~sum(1 << i for i in range(32) if (sel >> i) & 1 and rng.random() >= p_mid)
                    if not (sel & cand):
                        break
                mpr |= sel
    return passes


@pytest.mark.parametrize("wmode", [0, 1, 2])
def test_scan_passes_within_bound(wmode):
    rng = np.random.default_rng(wmode)
    worst = 0.0
    for _ in range(1500):
        Kadm = int(rng.integers(1, 257))
        S = int(rng.choice([2, 3, 16, 32, 64, 255, 256]))
        p_end, p_mid, p_ver = rng.uniform(0.3, 1.0), rng.uniform(0.3, 1.0), rng.uniform(0.0, 1.0)
        n = model_passes(rng, Kadm, S, wmode, p_end, p_mid, p_ver)
        cap = scan_pass_cap(Kadm, S)
        assert n <= cap, (Kadm, S, n, cap)
        worst = max(worst, n / cap)
    assert worst < 0.8


def test_bound_matches_the_kernel_formula():
    # the kernel's scan_pass_cap, read from its source
    import os
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2609_22608_gb300", "csrc",
                            "edge_core.cuh")).read()
    m = re.search(r"return \(\(n \+ 31\) / 32 \+ 1\) \* \(2 \+ 32 \* \(5 \+ \(S \+ 31\) / 32\)\) \+ 2;",
                  src)
    assert m, "scan_pass_cap changed: update the model's bound"
