"""Batched, uneven requests through the engine (dfp2s_engine_run): frames of different sizes, D/r0, J and
P2S form in one call, against the oracle's frames, the single-frame call and themselves across runs."""
import numpy as np
import pytest
import torch

from inputs import synthetic
from oracle import frame as oframe
from oracle import image, p2s, sampler

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as d
    d.load()
    return d


@pytest.fixture(scope="module")
def bases():
    return {J: p2s.build_basis(0, J, 16, 300, [1.0, 3.0, 5.0]) for J in (15, 36)}


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _handles(lib, bases):
    return {J: lib.P2S(J, torch.as_tensor(b, dtype=torch.float32, device="cuda")) for J, b in bases.items()}


def test_engine_uneven_requests_match_oracle(lib, bases):
    # (H, W, C, J): sizes and mode counts vary request to request, two frames each, all in one call
    shapes = [(24, 32, 3, 15), (40, 24, 1, 36), (33, 17, 3, 36), (16, 48, 2, 15), (20, 20, 3, 36), (24, 32, 3, 15)]
    rng = np.random.default_rng(17)
    P = _handles(lib, bases)
    eng = lib.Engine([P[15], P[36]])
    reqs = []
    for r, (H, W, C, J) in enumerate(shapes):
        img = synthetic.shapes(H, W, C, seed=r)
        reqs.append({"img": torch.as_tensor(img, device="cuda"), "J": J, "D_over_r0": float(rng.uniform(1.0, 5.0)),
                     "seed": 100 + r, "first_frame": 3 * r, "n_frames": 2, "mode": lib.P2S_EXACT,
                     "out": torch.full((2, C, H, W), float("nan"), device="cuda"), "np_img": img})
    eng.run(reqs)
    torch.cuda.synchronize()
    for r, q in enumerate(reqs):
        H, W, C, J = shapes[r]
        N = sampler.grid_size(H, W)
        for f in range(2):
            o = oframe.simulate_frame(q["np_img"], q["D_over_r0"], q["seed"], q["first_frame"] + f, J, bases[J],
                                      8.0, N)["out"]
            assert _rel(q["out"][f].cpu().numpy(), o) < TOL, (r, f)
    info = eng.info()
    assert info["frames"] == 12 and len(info["classes"]) == 5  # the first and last request share a class
    assert info["graph_launches"] == 5


def test_engine_frames_equal_single_frame_calls_and_graphs_update(lib, bases):
    P = _handles(lib, bases)
    eng = lib.Engine([P[36]])
    H, W, C = 48, 40, 3
    img = torch.as_tensor(synthetic.shapes(H, W, C, seed=4), device="cuda")
    out = torch.empty(3, C, H, W, device="cuda")
    req = {"img": img, "J": 36, "D_over_r0": 2.5, "seed": 9, "first_frame": 5, "n_frames": 3, "mode": lib.P2S_EXACT,
           "out": out}
    eng.run([req])
    first = out.clone()
    f = lib.SpectralFactor(36, sampler.grid_size(H, W), 8.0)
    sim = lib.Simulator(f, P[36], C, H, W)
    for k in range(3):
        assert torch.equal(sim.simulate_frame(img, 2.5, 9, 5 + k, lib.P2S_EXACT), first[k])
    # the same shape of work again: the class's graph is updated in place, the frames are the same bits
    out.zero_()
    eng.run([req])
    torch.cuda.synchronize()
    assert torch.equal(out, first)
    info = eng.info()
    assert info["graph_instantiations"] == 1 and info["graph_updates"] == 1
    # another seed: other frames
    req2 = dict(req, seed=10)
    eng.run([req2])
    assert not torch.equal(out, first)


def test_engine_learned_requests_and_tuning_report(lib, bases):
    J, K = 36, 16
    P = lib.P2S(J, torch.as_tensor(bases[J], dtype=torch.float32, device="cuda"))
    rng = np.random.default_rng(3)
    cu = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float32), device="cuda")
    shift = p2s.weights(np.zeros(J), J, bases[J])
    P.set_mlp(cu(rng.standard_normal((256, J)) / 6), cu(np.zeros(256)), cu(rng.standard_normal((256, 256)) / 16),
              cu(np.zeros(256)), cu(rng.standard_normal((K, 256)) / 16), cu(np.zeros(K)),
              cu(np.r_[0.0, 0.0, np.ones(J - 2)]), cu(np.full(K, 0.02)), cu(shift))
    eng = lib.Engine([P])
    reqs = []
    for r, (H, W) in enumerate([(64, 64), (96, 80), (64, 64)]):
        reqs.append({"img": torch.as_tensor(synthetic.shapes(H, W, 3, seed=r), device="cuda"), "J": J,
                     "D_over_r0": 2.0, "seed": r, "n_frames": 2, "mode": lib.P2S_LEARNED,
                     "out": torch.empty(2, 3, H, W, device="cuda")})
    eng.run(reqs)
    torch.cuda.synchronize()
    P.check()
    f = lib.SpectralFactor(J, 128, 8.0)
    sim = lib.Simulator(f, P, 3, 96, 80)
    for q in reqs:
        for k in range(2):
            assert torch.equal(sim.simulate_frame(q["img"], 2.0, q["seed"], k, lib.P2S_LEARNED), q["out"][k])
    for c in eng.info()["classes"]:
        assert c["column_pass"] in (0, 1)
        assert c["tuned_ms"][0] > 0 and c["tuned_ms"][1] > 0  # both candidates timed (N = 128)
        assert c["tuned_ms"][c["column_pass"]] == min(c["tuned_ms"])


def test_engine_mixed_grid_sizes_sampled_against_oracle(lib, bases):
    # the batched workload's image sides (256 .. 1024, grids 512 .. 2048) in one call, exact P2S, one frame per
    # request; the oracle at sampled pixels (fields on the full grid, warp, per-pixel exact weights, blur sum)
    P = _handles(lib, bases)
    eng = lib.Engine([P[15], P[36]])
    specs = [(256, 15, 1.3), (512, 36, 4.6), (768, 36, 2.2), (1024, 15, 3.7)]
    reqs = []
    for r, (side, J, dr) in enumerate(specs):
        img = synthetic.shapes(side, side, 3, seed=20 + r)
        reqs.append({"img": torch.as_tensor(img, device="cuda"), "J": J, "D_over_r0": dr, "seed": 50 + r,
                     "first_frame": r, "n_frames": 1, "mode": lib.P2S_EXACT,
                     "out": torch.empty(1, 3, side, side, device="cuda"), "np_img": img})
    eng.run(reqs)
    torch.cuda.synchronize()
    u = np.arange(-16, 17)
    for r, (side, J, dr) in enumerate(specs):
        q = reqs[r]
        N = sampler.grid_size(side, side)
        a = sampler.sample_fields(q["seed"], q["first_frame"], J, side, side, dr, 8.0, N)
        warped = image.tilt_warp(q["np_img"], a[0], a[1])
        g = q["out"][0].cpu().numpy()
        rng = np.random.default_rng(r)
        pts = [(0, 0), (side - 1, side - 1), (3, side - 2)] + [tuple(p) for p in rng.integers(0, side, (9, 2))]
        got, ref = [], []
        for y, x in pts:
            w = p2s.weights(a[:, y, x], J, bases[J])
            win = warped[:, np.clip(y - u, 0, side - 1)][:, :, np.clip(x - u, 0, side - 1)]
            ref.append((win * np.tensordot(w, bases[J], axes=1)[None]).sum(axis=(1, 2)))
            got.append(g[:, y, x])
        assert _rel(np.array(got), np.array(ref)) < TOL, (side, J)
