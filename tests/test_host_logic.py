"""Host-side planning (no GPU): Table 2 image sides by frequency, size-class runs of a band,
and the mixed stream's interleaving."""
import numpy as np

import synth


def test_image_side_follows_table2():
    import paper_1712_06913_b300 as m
    # Table 2: 0.4-0.6 GHz 256, 0.6-1.2 512, 1.2-2.0 1024, 2-4 1280, 4-8 2560, 8-15 5120
    f = np.array([0.4, 0.5999, 0.6, 1.1999, 1.2, 1.9999, 2.0, 3.9999, 4.0, 7.9999, 8.0, 15.0]) * 1e9
    assert m.image_side(f).tolist() == [256, 256, 512, 512, 1024, 1024, 1280, 1280, 2560, 2560, 5120, 5120]
    assert m.image_side(f, n_max=512).max() == 512


def test_size_classes_cover_the_band_in_runs():
    import paper_1712_06913_b300 as m
    for freq, n_max in ((synth.muser1_channels(), 512), (synth.muser2_channels(), 5120), (synth.muser2_channels(), 1024)):
        runs = m.size_classes(freq, n_max)
        assert runs[0][0] == 0 and runs[-1][1] == len(freq)
        assert all(a[1] == b[0] for a, b in zip(runs, runs[1:]))
        assert all(a[2] != b[2] for a, b in zip(runs, runs[1:]))
        for c0, c1, N in runs:
            assert set(m.image_side(freq[c0:c1], n_max).tolist()) == {N}
    assert [r[2] for r in m.size_classes(synth.muser1_channels(), 512)] == [256, 512]
    assert [r[2] for r in m.size_classes(synth.muser2_channels(), 5120)] == [1280, 2560, 5120]


def test_mixed_stream_order_covers_each_instance_once():
    w1, w2, order = synth.config5_mixed_stream(n_total=1200)
    assert len(order) == 1200
    assert sorted(i for s, i in order if s == 0) == list(range(600))
    assert sorted(i for s, i in order if s == 1) == list(range(600))
    assert order[0][0] == 0 and any(s == 1 for s, _ in order[:600])
