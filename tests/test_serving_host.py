"""Host-side parts of the serving loop (no GPU): the request stream and the latency summary."""
import math

import numpy as np

from paper_2407_13950_gb300 import serving
from paper_2407_13950_gb300 import synthetic as S


def test_poisson_stream_is_seeded_sorted_and_has_the_rate():
    sessions = [S.config_2q(), S.config_3q()]
    a = serving.poisson_requests(sessions, rate=500.0, duration=4.0, seed=3)
    b = serving.poisson_requests(sessions, rate=500.0, duration=4.0, seed=3)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(x.arrival <= y.arrival for x, y in zip(a, a[1:]))
    assert abs(len(a) - 2000) < 5 * math.sqrt(2000)          # Poisson count, 5 sigma
    frac = np.mean([r.gradient for r in a])
    assert abs(frac - 0.5) < 0.05
    for r in a[:20]:
        sp = sessions[r.session]
        assert r.alpha.shape == (sp.d,) and r.W.shape == (sp.nW,)


def test_latency_summary():
    reqs = [serving.Request(session=0, gradient=True, alpha=None, W=None, arrival=0.0, ready=0.5, done=1.0 + i)
            for i in range(100)]
    lat = serving.latency_summary(reqs)
    assert abs(lat["from_arrival"]["p50"] - 1000 * np.percentile(1.0 + np.arange(100), 50)) < 1e-6
    assert lat["from_ready"]["p99"] < lat["from_arrival"]["p99"]
