"""Checkpointed image libraries (paper_2302_02733_gb300/library.py) on the CPU: an interrupted
run resumes by skipping the finished ids, a torn record or a damaged image is rendered again,
and the finished library equals an uninterrupted one."""
import os

import numpy as np
import pytest

from paper_2302_02733_gb300.library import DONE, LibraryJob, finished_ids, render_library


class Cam:
    def __init__(self, n):
        self.nx = self.ny = n


def fake_image(job):
    rng = np.random.default_rng(job.id)
    return rng.random((job.camera.ny, job.camera.nx, 4))


def jobs(n=23):
    return [LibraryJob(id=100 + k, camera=Cam(4 + k % 3), M_unit=1e19, R_high=40.0) for k in range(n)]


class Interrupt(Exception):
    pass


def renderer(log, fail_after=None):
    def render(part):
        out = []
        for j in part:
            if fail_after is not None and len(log) >= fail_after:
                raise Interrupt()
            log.append(j.id)
            out.append(fake_image(j))
        return out
    return render


def test_interrupted_library_resumes(tmp_path):
    lib = jobs()
    log = []
    with pytest.raises(Interrupt):
        render_library(lib, str(tmp_path), renderer(log, fail_after=11), batch=5)
    # the batch in which the interruption fell is lost; the earlier ones are recorded
    assert finished_ids(str(tmp_path)) == {j.id for j in lib[:10]}
    log2 = []
    rendered = render_library(lib, str(tmp_path), renderer(log2), batch=5)
    assert rendered == log2 == [j.id for j in lib[10:]]
    assert render_library(lib, str(tmp_path), renderer([]), batch=5) == []
    ref = tmp_path / "ref"
    render_library(lib, str(ref), renderer([]), batch=7)
    for j in lib:
        name = f"img_{j.id:06d}.npy"
        assert np.array_equal(np.load(tmp_path / name), np.load(ref / name))


def test_damaged_records_are_rendered_again(tmp_path):
    lib = jobs(6)
    render_library(lib, str(tmp_path), renderer([]), batch=4)
    # a damaged image, a removed one, and a line cut short
    with open(tmp_path / f"img_{lib[1].id:06d}.npy", "r+b") as f:
        f.seek(-8, os.SEEK_END)
        f.write(b"\x00" * 8)
    os.remove(tmp_path / f"img_{lib[3].id:06d}.npy")
    with open(tmp_path / DONE, "a") as f:
        f.write(f"{lib[5].id} img_")
    log = []
    assert render_library(lib, str(tmp_path), renderer(log), batch=4) == [lib[1].id, lib[3].id]
    assert finished_ids(str(tmp_path)) == {j.id for j in lib}


def test_duplicate_ids_are_refused(tmp_path):
    lib = jobs(3) + [LibraryJob(id=100, camera=Cam(4))]
    with pytest.raises(ValueError):
        render_library(lib, str(tmp_path), renderer([]))
