"""Image libraries that survive interruption: checkpointed batched rendering.

The paper's motivation for fast images is the image library and the MCMC fit (Sections 1 and
4): thousands of images of different cameras and model parameters. A long library run that is
interrupted (a node lost, a job killed at its time limit) should not start over. This module
renders a library through rt_render_batch in batches and records each finished image:

* every finished image is written to ``<outdir>/img_<id>.npy`` (written to a temporary name and
  renamed, so a file that exists is complete);
* then its id, file name and SHA-256 are appended to ``<outdir>/done.txt`` and flushed;
* a restarted run reads done.txt and skips every id whose file exists with the recorded hash.
  An id listed but missing or corrupt is rendered again.

Images are rendered in the order of the job list, ``batch`` at a time; the rendering itself is a
callback (by default one rt_render_batch of the batch through the C ABI), so the bookkeeping
runs and is tested on the CPU.
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass
from typing import Callable, Sequence

import numpy as np

DONE = "done.txt"


@dataclass
class LibraryJob:
    """One image of a library: its id (unique in the library), camera and model parameters."""
    id: int
    camera: object      # a camera as for rt_set_camera (nx, ny, incl_deg, ...)
    M_unit: float = 0.0  # 0: the loaded model's
    R_high: float = 0.0


def _digest(path: str) -> str:
    h = hashlib.sha256()
    with open(path, "rb") as f:
        for chunk in iter(lambda: f.read(1 << 20), b""):
            h.update(chunk)
    return h.hexdigest()


def finished_ids(outdir: str) -> set[int]:
    """Ids recorded in done.txt whose image file exists with the recorded hash."""
    done = set()
    path = os.path.join(outdir, DONE)
    if not os.path.exists(path):
        return done
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) != 3:
                continue  # a line cut short by the interruption
            try:
                jid = int(parts[0])
            except ValueError:
                continue
            img = os.path.join(outdir, parts[1])
            if os.path.exists(img) and _digest(img) == parts[2]:
                done.add(jid)
    return done


def _save(outdir: str, jid: int, image: np.ndarray) -> None:
    name = f"img_{jid:06d}.npy"
    tmp = os.path.join(outdir, name + ".part")
    with open(tmp, "wb") as f:
        np.save(f, image)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, os.path.join(outdir, name))
    with open(os.path.join(outdir, DONE), "a") as f:
        f.write(f"{jid} {name} {_digest(os.path.join(outdir, name))}\n")
        f.flush()
        os.fsync(f.fileno())


def render_library(jobs: Sequence[LibraryJob], outdir: str, render_batch: Callable[[list], list],
                   batch: int = 16) -> list[int]:
    """Render the jobs not yet finished in outdir, ``batch`` at a time.

    render_batch(list of LibraryJob) -> list of images (numpy arrays), one per job, in order.
    Returns the ids rendered by this call (the others were skipped as finished)."""
    ids = [j.id for j in jobs]
    if len(set(ids)) != len(ids):
        raise ValueError("library job ids must be unique")
    os.makedirs(outdir, exist_ok=True)
    done = finished_ids(outdir)
    todo = [j for j in jobs if j.id not in done]
    rendered = []
    for k in range(0, len(todo), batch):
        part = todo[k:k + batch]
        images = render_batch(part)
        if len(images) != len(part):
            raise RuntimeError("render_batch returned the wrong number of images")
        for j, img in zip(part, images):
            _save(outdir, j.id, np.asarray(img))
            rendered.append(j.id)
    return rendered


def gpu_batch_renderer(ctx, form: int, device: str = "cuda"):
    """The default render_batch: one rt_render_batch of the batch on ctx (the loaded model),
    images copied back to host memory."""
    import torch

    from paper_2302_02733_gb300 import polrt

    dt = torch.float64 if form == polrt.RT_FP64 else torch.float32

    def render(part):
        shape = (lambda c: (c.ny, c.nx) if form == polrt.RT_UNPOL else (c.ny, c.nx, 4))
        outs = [torch.empty(shape(j.camera), dtype=dt, device=device) for j in part]
        table = polrt.make_jobs((j.camera, j.M_unit, j.R_high, o, None, None) for j, o in zip(part, outs))
        polrt.rt_render_batch(ctx, form, table)
        return [o.cpu().numpy() for o in outs]

    return render
