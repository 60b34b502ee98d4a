"""Test-side stand-in for the library's D3Q27 sweep on CPU: the AA-pattern
sweep over the active planes of a local grid, each node collided by the FP64
oracle (test infrastructure only; the product's sweeps are CUDA kernels).

Even sweep: node x reads slot (x, i) as f_i, writes f*_i to slot (x, opp(i)).
Odd sweep: node x reads f_opp(j) from slot (x + e_j, j), writes f*_j there.
Slots are periodic in x and y, not wrapped in z (ghost planes lie outside the
active range)."""
import numpy as np

import oracle

def velocities():
    return np.array([[(i // 3 ** d) % 3 - 1 for d in range(3)] for i in range(27)])


def opp(i):
    return 26 - i


class OracleAASim:
    def __init__(self, dims, omega, z_lo, z_cnt, torch):
        self.nx, self.ny, self.nz = dims
        self.omega = np.asarray(omega, dtype=np.float64)
        self.z_lo, self.z_cnt = z_lo, z_cnt
        self.N = self.nx * self.ny * self.nz
        self.pop = torch.zeros(27, self.N, dtype=torch.float64)
        self.step_count = 0
        self.e = velocities()

    def raw_populations(self):
        return self.pop

    def init_natural(self, f):
        """Even-state layout: slot (x, i) = f_i(x)."""
        self.pop.copy_(self.pop.new_tensor(np.asarray(f)))
        self.step_count = 0

    def _node(self, x, y, z):
        return x + self.nx * (y + self.ny * z)

    def _slot(self, x, y, z, j):
        e = self.e[j]
        xn, yn, zn = (x + e[0]) % self.nx, (y + e[1]) % self.ny, z + e[2]
        assert 0 <= zn < self.nz
        return self._node(xn, yn, zn)

    def step(self, n=1):
        P = self.pop.numpy()
        for _ in range(n):
            odd = self.step_count & 1
            for z in range(self.z_lo, self.z_lo + self.z_cnt):
                for y in range(self.ny):
                    for x in range(self.nx):
                        if not odd:
                            k = self._node(x, y, z)
                            f = P[:, k].copy()
                            post = oracle.tp_collide_node(3, self.omega, f, oracle.ORC_KRONECKER)
                            for i in range(27):
                                P[opp(i), k] = post[i]
                        else:
                            slots = [self._slot(x, y, z, j) for j in range(27)]
                            f = np.empty(27)
                            for j in range(27):
                                f[opp(j)] = P[j, slots[j]]
                            post = oracle.tp_collide_node(3, self.omega, f, oracle.ORC_KRONECKER)
                            for j in range(27):
                                P[j, slots[j]] = post[j]
            self.step_count += 1


def natural_from_aa(P, dims, odd):
    """Populations f_i(x) of a whole periodic grid from its AA buffer."""
    if not odd:
        return np.array(P, copy=True)
    nx, ny, nz = dims
    e = velocities()
    out = np.empty_like(P)
    idx = np.arange(nx * ny * nz)
    x, y, z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    for k in range(27):
        # population k of node x sits in slot (x - e_k, opp(k))
        xs, ys, zs = (x - e[k, 0]) % nx, (y - e[k, 1]) % ny, (z - e[k, 2]) % nz
        out[k] = P[opp(k), xs + nx * (ys + ny * zs)]
    return out
