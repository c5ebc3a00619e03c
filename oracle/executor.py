"""Sequential oracle executor: the task model with the runtime taken away.

TEST INFRASTRUCTURE ONLY.

Section 2 of the paper: a task is declared with its implementations, its
number of buffers and one access mode per buffer; buffers are registered
before use; an invocation is asynchronous and a wait joins all pending
tasks.  Section 3: with the annotations ignored the program is a valid
sequential program.  This executor keeps the same four calls but runs every
task at the moment it is submitted, in submission order, so its results are
the reference the device executor must reproduce.

It also records each task's accesses, so the dependency oracle (dag.py)
can derive the graph the device executor is expected to build.
"""
import numpy as np

from . import tiles as _t
from .dag import R, W, RW


class OracleError(Exception):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


ENOENT, EINVAL = 2, 22


class Executor:
    def __init__(self):
        self.codelets = []
        self.buffers = []
        self.by_addr = {}
        self.accesses = []
        self.names = []

    # Section 2: the codelet names the task, its buffers and their modes.
    def task_decl(self, name, impl, modes, scalar_bytes=0):
        self.codelets.append((name, impl, tuple(modes), scalar_bytes))
        return len(self.codelets) - 1

    # Section 2: buffers are registered before tasks use them.
    def data_register(self, array):
        h = len(self.buffers)
        self.buffers.append(array)
        self.by_addr[array.__array_interface__["data"][0]] = h
        return h

    # Section 3.2: an unregistered pointer is an error.
    def data_lookup(self, array):
        h = self.by_addr.get(array.__array_interface__["data"][0])
        if h is None:
            raise OracleError(ENOENT, "attempt to use unregistered pointer")
        return h

    def task_submit(self, codelet, handles, modes=None, scalars=()):
        name, impl, cmodes, _ = self.codelets[codelet]
        modes = tuple(modes) if modes is not None else cmodes
        if len(handles) != len(cmodes) or modes != cmodes:
            raise OracleError(EINVAL, "task/implementation signature mismatch")
        for h in handles:
            if not (0 <= h < len(self.buffers)):
                raise OracleError(ENOENT, "unregistered handle")
        self.accesses.append(list(zip(handles, modes)))
        self.names.append(name)
        impl(*[self.buffers[h] for h in handles], *scalars)

    def task_wait(self):
        return 0


# Task bodies (Section 2 example and the tile kernels of the Cholesky idiom).
def scal_body(x, f):
    _t.scal_f32(x, np.float32(f))


def noop_body(*bufs):
    pass
