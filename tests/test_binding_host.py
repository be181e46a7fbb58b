"""The Python binding's argument checks, on the CPU.

The binding only marshals arguments; what it refuses it refuses before any
call into libtc: edge arrays that are not contiguous 1-D int32 (CUDA tensors
for the device calls; numpy arrays or CPU tensors for the host calls),
length mismatches, mis-sized outputs and batch offsets that do not match
their vertex counts.  Status codes the library returns become TCError with
the code and the library's detail string."""
import numpy as np
import pytest
import torch

import paper_1503_00576_gb300 as tc

pytestmark = pytest.mark.usefixtures("libtc")


def i32(*x):
    return torch.tensor(x, dtype=torch.int32)


def test_device_calls_want_cuda_int32():
    with pytest.raises(TypeError, match="CUDA tensor"):
        tc.tc_count(i32(0, 1), i32(1, 2), 3)
    with pytest.raises(TypeError, match="CUDA tensor"):
        tc.tc_count(np.array([0, 1], np.int32), np.array([1, 2], np.int32), 3)
    with pytest.raises(TypeError, match="CUDA tensor"):
        tc.tc_count_per_vertex(i32(0), i32(1), 2)
    with pytest.raises(TypeError, match="CUDA tensor"):
        tc.tc_count_batch(i32(0), i32(1), [0, 1], [2])
    with pytest.raises(TypeError, match="CUDA tensor"):
        tc.tc_count_work(i32(0), i32(1), 2)


def test_host_calls_want_contiguous_int32():
    with pytest.raises(TypeError, match="int32"):
        tc.tc_count_host(np.array([0, 1], np.int64), np.array([1, 2], np.int32), 3)
    with pytest.raises(TypeError, match="int32"):
        tc.tc_count_host(np.arange(6, dtype=np.int32)[::2], np.arange(3, dtype=np.int32), 6)
    with pytest.raises(TypeError, match="int32"):
        tc.tc_count_host(torch.zeros(3, dtype=torch.int64), i32(0, 1, 2), 3)
    with pytest.raises(ValueError, match="differ in length"):
        tc.tc_count_host(np.zeros(3, np.int32), np.zeros(2, np.int32), 3)
    with pytest.raises(TypeError, match="8-byte items"):
        tc.tc_count_per_vertex_host(np.zeros(2, np.int32), np.ones(2, np.int32), 2,
                                    t_out=np.zeros(2, np.int32))
    with pytest.raises(TypeError, match="numpy array or a contiguous CPU tensor"):
        tc.tc_count_per_vertex_host(np.zeros(2, np.int32), np.ones(2, np.int32), 2,
                                    t_out=[0, 0])


def test_batch_offsets_match_counts():
    with pytest.raises(ValueError, match="one entry more"):
        tc._batch_arrays([0, 3], [4, 5])
    with pytest.raises(ValueError, match="one entry more"):
        tc._batch_arrays(np.zeros((2, 2)), [1])
    eo, vn = tc._batch_arrays([0, 3, 3], [4, 1])
    assert eo.dtype == np.int64 and vn.dtype == np.int32 and list(eo) == [0, 3, 3]


def test_status_codes_become_errors():
    with pytest.raises(tc.TCError) as e:
        tc.tc_set_tuning({"heavy_ratio_pct": 50})
    assert e.value.code == tc.TC_ERR_INVALID_ARG
    assert "tuning" in e.value.detail and "invalid argument" in str(e.value)
    with pytest.raises(tc.TCError) as e:
        tc.tc_set_tuning({"hub_vertices": 1000})  # not a multiple of 128
    assert e.value.code == tc.TC_ERR_INVALID_ARG
    assert tc.tc_get_tuning() == tc.DEFAULT_TUNING  # a refused tuning changes nothing


def test_workspace_bytes_through_the_binding():
    assert tc.tc_workspace_bytes(0, 0) > 0
    assert tc.tc_workspace_bytes(10 ** 6, 10 ** 5) > 16 * 10 ** 6
    assert tc.tc_workspace_bytes(1 << 31, 5) == 0


@pytest.mark.parametrize("spec,want", [('{"heavy_ratio_pct": 150, "warp_max_list": 64}', 0),
                                       ('{"hub_vertices": 1000}', 1)])
def test_tuning_from_the_environment(spec, want):
    """TC_TUNING sets the process-wide tuning when the library loads; a
    value the library refuses raises there."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import paper_1503_00576_gb300 as tc\n"
            "try:\n"
            "    tc.load_library()\n"
            "except tc.TCError as e:\n"
            "    raise SystemExit(e.code)\n"
            "t = tc.tc_get_tuning()\n"
            "assert t['heavy_ratio_pct'] == 150 and t['warp_max_list'] == 64, t\n"
            "assert t['hub_vertices'] == tc.DEFAULT_TUNING['hub_vertices']\n")
    env = dict(os.environ, TC_TUNING=spec)
    rc = subprocess.run([sys.executable, "-c", code], cwd=root, env=env).returncode
    assert rc == want
