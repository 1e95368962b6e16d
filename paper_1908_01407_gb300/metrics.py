"""Host-side metric arithmetic (no device work)."""


def teps(m_stored: int, seconds: float) -> float:
    """Traversed edges per second as the paper reports it: the stored
    (symmetrised) nonzeros of A over the runtime (Section 8, measurement
    methodology; Table 12's rmat_s22_e64 row: 483M / 4.781 ms = 101 GTEPS)."""
    return m_stored / seconds


def teps_undirected(m_stored: int, seconds: float) -> float:
    """Graph500 convention: undirected edges (half the stored nonzeros)."""
    return (m_stored / 2) / seconds
