"""Host logic of the autotuner (CPU, with a fake timer)."""
from paper_2604_03092_gb300 import autotune, scenes


def test_tune_picks_fastest_and_caches(tmp_path):
    sc = scenes.random_scene(n=1000, width=64, height=48, f=50.0, seed=0, n_views=2)
    path = str(tmp_path / "cache.json")
    calls = []

    def fake(c):
        calls.append(c)
        return {(8, 8, 128): 1.5}.get(c, 2.0 + c[2] / 1000)

    best, res = autotune.tune(sc.views, sc.n, fake, path=path)
    assert best == (8, 8, 128)
    assert len(calls) == len(autotune.CANDIDATES) and len(res) == len(calls)
    assert autotune.lookup(sc.views, sc.n, path=path) == (8, 8, 128)
    # cached: no re-timing
    best2, _ = autotune.tune(sc.views, sc.n, lambda c: 1 / 0, path=path)
    assert best2 == (8, 8, 128)
    # a different bucket is not served from the cache
    big = scenes.random_scene(n=1000, width=640, height=480, f=500.0, seed=0)
    assert autotune.lookup(big.views, big.n, path=path) is None


def test_bucket_key_separates_image_size_and_density():
    a = scenes.random_scene(n=1000, width=64, height=48, seed=0)
    b = scenes.random_scene(n=100000, width=64, height=48, seed=0, with_target=False)
    c = scenes.random_scene(n=1000, width=512, height=384, seed=0, with_target=False)
    ka, kb, kc = (autotune.bucket_key(s.views, s.n) for s in (a, b, c))
    assert len({ka, kb, kc}) == 3
