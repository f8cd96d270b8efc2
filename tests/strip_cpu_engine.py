"""A CPU stand-in for one strip's GPU work in the row-strip tests: the
paper's layer rule written on distances (Methods, "Activity Map
Generation"): at layer l an unreached free cell with an 8-neighbour at l - 1
is reached at l. Test infrastructure only (the product runs the library)."""
import numpy as np

INF = 0xFFFFFFFF


class CpuStripEngine:
    device = None

    def __init__(self, ext_mask):
        self.free = np.asarray(ext_mask) == 0

    def resume(self, plane, frm, to):
        d = np.where(np.asarray(plane) <= frm, plane, INF).astype(np.uint32)
        H, W = d.shape
        for l in range(frm + 1, to + 1):
            prev = np.zeros((H + 2, W + 2), bool)
            prev[1:-1, 1:-1] = d == l - 1
            near = np.zeros((H, W), bool)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dy or dx:
                        near |= prev[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            new = near & self.free & (d == INF)
            if not new.any():
                break
            d[new] = l
        return d
