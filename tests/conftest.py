import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def cfg1():
    import synth
    return synth.uplift_cfg1()


@pytest.fixture(scope="session")
def cfg1_oracle(oracle_lib, cfg1):
    acc, risk, cnt = oracle_lib.uplift(cfg1)
    idx, val = oracle_lib.topk(acc, cfg1.K)
    return {"acc": acc, "risk": risk, "counts": cnt, "idx": idx, "val": val}


def axis_camera(width=64, height=48, f=50.0, cx=None, cy=None, z=0.0, R=None):
    """Camera with world->camera rotation R (default identity) and translation
    (0, 0, z): a point at world origin lands at camera depth z."""
    import synth
    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    vm = np.concatenate([R, np.array([[0.0], [0.0], [z]])], axis=1).reshape(12)
    return synth.Camera(vm.astype(np.float32), float(f), float(f),
                        float(width / 2.0 if cx is None else cx),
                        float(height / 2.0 if cy is None else cy), int(width), int(height))


def make_scene(means, scales, quats, opacity):
    import synth
    return synth.Scene(np.asarray(means, np.float32).reshape(-1, 3),
                       np.asarray(scales, np.float32).reshape(-1, 3),
                       np.asarray(quats, np.float32).reshape(-1, 4),
                       np.asarray(opacity, np.float32).reshape(-1))


def single_region_workload(scene, cams, C, code_pairs, K, name="custom"):
    """All pixels of every view in region 0 with code [(atom, value), ...]."""
    import synth
    maps, offs = [], [0]
    for c in cams:
        maps.append(np.zeros(c.width * c.height, np.int32))
        offs.append(offs[-1] + c.width * c.height)
    s = len(code_pairs)
    ci = np.array([[a for a, _ in code_pairs]], np.int32)
    cv = np.array([[v for _, v in code_pairs]], np.float32)
    return synth.UpliftWorkload(name, scene, list(cams), np.concatenate(maps),
                                np.array(offs, np.int64), ci, cv, C, s, K, [1] * len(cams))
