"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point declared in include/maxsat.h, validates arguments
before touching the device, and fits OR-gate RBMs on the host."""
import ctypes
import itertools
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2311_02101_gb300 as ms
from paper_2311_02101_gb300 import build as msbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    msbuild.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "maxsat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(maxsat_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert "maxsat_create" in names and "maxsat_step" in names and len(names) >= 13
    L = ctypes.CDLL(msbuild.LIB)
    for name in names:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", msbuild.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (maxsat_\w+)", out))
    assert set(names) <= exported
    assert exported <= set(names), exported - set(names)  # nothing undeclared


def test_default_params():
    p = ms.maxsat_default_params()
    assert (p.n_temps, p.n_buckets, p.quant_bits, p.path, p.fit_iters, p.steps_per_graph) == \
        (2, 4, 4, ms.MAXSAT_PATH_AUTO, 50000, 100)
    assert p.alpha == 0.01 and p.bucket_gamma == 0.5 and not p.fstar and p.n_sets == 0
    assert (p.tune_blocks, p.up_device, p.visible_batch, p.persistent_round) == (0, 1, 0, 0)


@pytest.mark.parametrize("K,fs", [(2, 0.528), (3, 0.068), (3, 0.528), (5, 0.528)])
def test_library_fit_reaches_or_target(K, fs):
    """Sec. 4.1: the fitted clause free energy is ~0 on the all-false input
    and ~F_s = -F* elsewhere; W lies on the 2^-4 grid and b on the 2^-24 grid."""
    L = 3 if K <= 3 else K + 1
    W, b = ms.maxsat_fit_or_rbm(K, L, fs, 4, 50000)
    assert np.all(W * 16 == np.round(W * 16))
    assert np.all(b * 2 ** 24 == np.round(b * 2 ** 24))
    V = np.array(list(itertools.product([0.0, 1.0], repeat=K)))
    F = -np.logaddexp(0, V @ W + b).sum(axis=1)
    assert abs(F[0]) < 0.06
    assert np.max(np.abs(F[1:] + fs)) < 0.08


def test_fit_rejects_bad_arguments():
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_fit_or_rbm(13, 3, 0.5)
    assert e.value.code == ms.MAXSAT_EINVAL
    with pytest.raises(ms.MaxsatError):
        ms.maxsat_fit_or_rbm(3, 17, 0.5)


@pytest.mark.parametrize("n,off,lits,w,msg", [
    (0, [0, 1], [1], None, "n_vars"),
    (3, [1, 2], [1, 2], None, "clause_off[0]"),
    (3, [0, 2, 1], [1, 2], None, "non-decreasing"),
    (3, [0, 2], [1, 4], None, "out of range"),
    (3, [0, 2], [1, 0], None, "out of range"),
    (3, [0, 2], [1, 2], [0], "weights"),
    (13, [0, 13], list(range(1, 14)), None, "MAXSAT_MAX_LEN"),
])
def test_create_validates_before_device(n, off, lits, w, msg):
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_create(n, off, lits, w)
    assert e.value.code == ms.MAXSAT_EINVAL
    assert msg in str(e.value)


@pytest.mark.parametrize("insts,msg", [
    ([(0, [0, 1], [1], None)], "n_vars >= 1"),
    ([(3, [0, 2], [1, 2], None), (2, [0, 1], [3], None)], "instance 1: literal"),
    ([(3, [0, 2], [1, -4], None)], "instance 0: literal"),
    ([(3, [0, 2], [1, 2], [0])], "weights"),
    ([(13, [0, 13], list(range(1, 14)), None)], "MAXSAT_MAX_LEN"),
])
def test_create_batch_validates_before_device(insts, msg):
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_create_batch(insts)
    assert e.value.code == ms.MAXSAT_EINVAL
    assert msg in str(e.value)


@pytest.mark.parametrize("field,value,msg", [
    ("persistent_round", 2, "persistent_round must be 0 or 1"),
    ("visible_batch", 3, "visible_batch must be 0, 2, 4 or 8"),
    ("steps_per_graph", -1, "steps_per_graph out of range"),
])
def test_params_are_validated_before_device(field, value, msg):
    p = ms.maxsat_default_params(**{field: value})
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_create(3, [0, 2], [1, -2], None, p)
    assert e.value.code == ms.MAXSAT_EINVAL and msg in str(e.value)


def test_create_batch_dense_path_is_rejected():
    p = ms.maxsat_default_params(path=ms.MAXSAT_PATH_DENSE)
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_create_batch([(3, [0, 2], [1, 2], None), (2, [0, 1], [-2], None)], p)
    assert e.value.code == ms.MAXSAT_EINVAL and "sparse path" in str(e.value)


def test_create_without_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_create(3, [0, 2], [1, -2])
    assert e.value.code == ms.MAXSAT_ENODEV
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_create_batch([(3, [0, 2], [1, -2], None), (2, [0, 1], [2], None)])
    assert e.value.code == ms.MAXSAT_ENODEV


def test_product_never_touches_the_oracle():
    """The CUDA library and its binding share nothing with the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2311_02101_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle|rbmsat_oracle|oracle/", text,
                                     re.M), f
