"""Host-side mirrors of small library constants (documentation and tests)."""

X_CLASS_UPPER = (15, 35, 75, 150, 300, 700, 2000, 1 << 29)


def x_class(X: int) -> int:
    """X class of the start-level table (same bounds as the library)."""
    for c, hi in enumerate(X_CLASS_UPPER):
        if X <= hi:
            return c
    return len(X_CLASS_UPPER) - 1
