"""Host-side logic of the streaming pipeline that needs no GPU: binding the process to the CPUs
next to a device (the sysfs topology parsed, the affinity restricted, nothing changed where the
topology is missing)."""
import os

import pytest

from paper_2504_14338_gb300 import graph


class _Props:
    pci_domain_id, pci_bus_id, pci_device_id = 0, 0x1B, 0


@pytest.fixture
def fake_topology(monkeypatch, tmp_path):
    calls = {}
    monkeypatch.setattr(graph.torch.cuda, "get_device_properties", lambda dev: _Props())
    monkeypatch.setattr(graph.torch, "device", lambda d: d)
    real_open = open

    def fake_open(path, *a, **k):
        if str(path).startswith("/sys/bus/pci/devices/"):
            calls["path"] = path
            return real_open(tmp_path / "local_cpulist", *a, **k)
        return real_open(path, *a, **k)

    monkeypatch.setattr("builtins.open", fake_open)
    monkeypatch.setattr(os, "sched_getaffinity", lambda pid: set(range(64)))
    monkeypatch.setattr(os, "sched_setaffinity", lambda pid, cpus: calls.__setitem__("set", set(cpus)))
    return tmp_path, calls


def test_cpu_list_is_parsed_and_applied(fake_topology):
    tmp, calls = fake_topology
    (tmp / "local_cpulist").write_text("0-3,8,10-11\n")
    assert graph.bind_host_to_device("cuda:0") == "0-3,8,10-11"
    assert calls["path"] == "/sys/bus/pci/devices/0000:1b:00.0/local_cpulist"
    assert calls["set"] == {0, 1, 2, 3, 8, 10, 11}


def test_only_cpus_already_allowed_are_kept(fake_topology):
    tmp, calls = fake_topology
    (tmp / "local_cpulist").write_text("60-70\n")
    assert graph.bind_host_to_device("cuda:0") == "60-70"
    assert calls["set"] == {60, 61, 62, 63}


def test_nothing_changes_without_topology(monkeypatch):
    def boom(dev):
        raise RuntimeError("no device")

    monkeypatch.setattr(graph.torch.cuda, "get_device_properties", boom)
    monkeypatch.setattr(os, "sched_setaffinity", lambda pid, cpus: pytest.fail("affinity changed"))
    assert graph.bind_host_to_device("cuda:0") is None


def test_disjoint_cpu_list_changes_nothing(fake_topology, monkeypatch):
    tmp, calls = fake_topology
    (tmp / "local_cpulist").write_text("100-101\n")
    assert graph.bind_host_to_device("cuda:0") is None
    assert "set" not in calls


def test_snapshots_torch_with_a_precomputed_trajectory():
    """The device-side generator gives the same matrix whether it integrates the generating
    system itself or is handed that trajectory (formed by another process), on the CPU."""
    import numpy as np
    import torch
    from paper_2504_14338_gb300 import synth
    w = synth.Workload("traj", 2, 64, 40, 5, seed=17)
    a = synth.snapshots_torch(w, "cpu")
    traj = synth.trajectory(w)
    b = synth.snapshots_torch(w, "cpu", traj=traj)
    assert torch.equal(a, b)
    assert np.array_equal(traj[0], synth.trajectory(w)[0])
