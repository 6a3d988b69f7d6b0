"""Host-side helpers of bench.py (no GPU): the CPU-list parser and the
placement of the end-to-end leg's page-locked buffers on the GPU's local
CPUs, against a fake device and a fake sysfs tree."""
import os
import types

import pytest

import bench


def test_parse_cpulist():
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()


@pytest.mark.skipif(not hasattr(os, "sched_setaffinity"), reason="no CPU affinity on this platform")
def test_pin_to_local_cpus(tmp_path, monkeypatch):
    import torch
    before = os.sched_getaffinity(0)
    first = min(before)
    props = types.SimpleNamespace(pci_domain_id=0, pci_bus_id=0x07, pci_device_id=0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: props)
    dev = tmp_path / "0000:07:00.0"
    dev.mkdir()
    try:
        (dev / "local_cpulist").write_text(f"{first}\n")
        assert bench.pin_to_local_cpus(0, sysfs=str(tmp_path)) == str(first)
        assert os.sched_getaffinity(0) == {first}
        # a list outside the allowed CPUs, or no list at all: nothing changes
        os.sched_setaffinity(0, before)
        (dev / "local_cpulist").write_text("100000-100001\n")
        assert bench.pin_to_local_cpus(0, sysfs=str(tmp_path)) is None
        assert os.sched_getaffinity(0) == before
        assert bench.pin_to_local_cpus(0, sysfs=str(tmp_path / "missing")) is None
        assert os.sched_getaffinity(0) == before
    finally:
        os.sched_setaffinity(0, before)
