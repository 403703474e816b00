"""The C ABI library builds for sm_103a, loads, and exports every function
that include/ssh.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

from paper_1610_07328_gb300 import binding, build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ssh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssh_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["ssh_create", "ssh_destroy", "ssh_index_add", "ssh_index_add_device", "ssh_query",
                     "ssh_query_device", "ssh_status_str"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)
    assert set(_declared()) == set(binding.EXPORTED)


def test_library_is_sm103a_and_in_tree():
    path = build_ext.build()
    assert path.startswith(os.path.join(ROOT, "paper_1610_07328_gb300"))
    assert "arch=compute_103a,code=sm_103a" in build_ext.ARCH


def test_status_strings():
    lib = binding.load()
    assert lib.ssh_status_str(0) == b"SSH_OK"
    assert lib.ssh_status_str(4) == b"SSH_ELENGTH"
    assert lib.ssh_status_str(99) == b"SSH_UNKNOWN"
